// LSQR (Paige & Saunders 1982) on the augmented problem of Eq. (augmented),
// Sec. 3:  min || [A; sqrt(gamma) D] delta - r0 ||,
//   r0 = [b - A x0; sqrt(gamma) (c - D x0)],
//   D = diag(w) L (IRLS, Alg. 1), D = L with shift c = w (MM, Alg. 2) or
//   c = d - g (SB, Alg. 3).
//
// One persistent cooperative launch runs whole solves for a batch of
// problems (any mix of levels, sizes and solvers). Each Golub-Kahan step is
// two fused passes over 32x32 tiles, separated by grid barriers:
//   pass F_i: delta/w update of step i-1, then u_{i+1} = A_hat v_i - alpha_i u_i,
//             with ||u_{i+1}||^2, ||delta_{i-1}||^2, ||w_{i-1}||^2;
//   pass B_i: v_{i+1} = A_hat^T u_{i+1} - beta_{i+1} v_i with ||v_{i+1}||^2.
// u and v are stored unnormalised (u~ = beta u, v~ = alpha v) and rescaled on
// load. Norms are summed per tile in double; the block that finishes the last
// tile of a problem reduces that problem's tile partials in a fixed order and
// runs the scalar recurrence and the stopping tests (rules S1-S3 with the
// usual estimates, ||delta|| computed exactly) in double.
#pragma once
#include "toep.cuh"

namespace db {

template <typename T, typename Acc>
struct LsqrProb {
  using X = typename Traits<T>::X;
  BandOp<Acc> op;
  int m, solver;                 // 0 IRLS (weighted D), 1 MM (c = a0), 2 SB (c = a0 - a1)
  double gamma;
  Acc sg;                        // sqrt(gamma) in working precision
  const T* b;
  const X* x0;                   // null: start from zero
  const T *a0x, *a0y, *a1x, *a1y;
  T *uA, *uLx, *uLy, *v, *w;
  X* dlt;
  int tile_begin, ntiles, nt;    // tiles [tile_begin, tile_begin + ntiles), nt per side
  // tensor maps of the window loads of the direct level-0 path (op.toep):
  // v (pass F), u~_A (pass B) and x0 (pass F of the first phase)
  const CUtensorMap* tm_v;
  const CUtensorMap* tm_u;
  const CUtensorMap* tm_x0;
};

struct LsqrState {
  double alpha, beta, rhobar, phibar, anorm2, dnorm2, bnorm;
  double phi_rho, theta_rho, irho_last, t_rnorm, t_arnorm;
  int it, done, its, stop;       // stop: 1 S1, 2 S2, 3 S3, 4 maxit, 5 zero rhs/A^T rhs
};

// Working-precision coefficients of the next pass, written once per problem
// by the block that finished the previous pass (so no thread repeats the
// double-precision divisions):
//   pass F: v = v~ * inv_alpha, u~_new = A_hat v - ab * u~, delta += phr w, w = v - thr w
//   pass B: u = u~ * inv_beta, v~_new = A_hat^T u - ba * v~
template <typename Acc>
struct LsqrCoef {
  Acc inv_alpha, ab, phr, thr, inv_beta, ba;
};

struct LsqrCtl {
  double atol, btol, conlim;
  int maxit, nprob, ntiles;
  const int* tile_prob;          // [ntiles] problem of each tile
  double* part;                  // [ntiles * 3] per-tile partial sums
  unsigned* cnt;                 // [nprob] tiles finished in the current phase
  LsqrState* st;                 // [nprob]
  void* coef;                    // [nprob] LsqrCoef<Acc>
  GridBarrier* gb;
  unsigned long long limit_ns;
  int band_cache;                // 1: band rows of the cached tiles kept in shared memory (one-term PSFs)
  int band_pw;                   // row pitch of the band cache (Acc elements)
  int cache_off;                 // offset of the band cache in dynamic shared memory (Acc elements)
};

template <typename T>
__device__ __forceinline__ typename Traits<T>::Acc ldcg(const T* p) { return gload<true, T>(p); }

__device__ __forceinline__ LsqrState load_state(const LsqrState* s) {
  LsqrState r;
  const double* d = reinterpret_cast<const double*>(s);
  double* o = reinterpret_cast<double*>(&r);
#pragma unroll
  for (int k = 0; k < 12; ++k) o[k] = __ldcg(d + k);
  const int* di = reinterpret_cast<const int*>(d + 12);
  int* oi = reinterpret_cast<int*>(o + 12);
#pragma unroll
  for (int k = 0; k < 4; ++k) oi[k] = __ldcg(di + k);
  return r;
}

// The three per-thread sums of squares of a pass. For float working
// precision each sum is a double-float pair and each square enters exactly
// (its rounding error recovered with one FMA), so the tile partials carry
// about twice float precision; for double working precision, plain doubles.
template <typename Acc> struct Sums3;
template <> struct Sums3<float> {
  float h[3] = {0.f, 0.f, 0.f}, l[3] = {0.f, 0.f, 0.f};
  __device__ __forceinline__ void sq(int k, float a) { df_fma(h[k], l[k], a, a); }
};
template <> struct Sums3<double> {
  double h[3] = {0.0, 0.0, 0.0};
  __device__ __forceinline__ void sq(int k, double a) { h[k] = fma(a, a, h[k]); }
};

__device__ int lsqr_wait_release(const LsqrCtl& ctl, int ph);

// The waits read the clock every 64 spins, or on every spin when the limit is
// below 100 us (so that a short limit is honoured).
__device__ __forceinline__ unsigned spin_mask(const LsqrCtl& ctl) { return ctl.limit_ns < 100000ull ? 0u : 63u; }

// Loads of one tile issued before any of them is used: the problem's done
// flag and coefficients, the pointwise operands of this thread's pixels, the
// (unscaled) input window and the band rows of term 0. A pass then waits on
// a single memory round trip instead of a chain of them. The scale of the
// input (1/alpha or 1/beta) is applied to the outputs, which are linear in it.
template <typename Acc>
struct TileHead {
  int done;
  LsqrCoef<Acc> K;
};

template <typename Acc>
__device__ __forceinline__ TileHead<Acc> load_head(const LsqrCtl& ctl, int p) {
  TileHead<Acc> h;
  h.done = __ldcg(&ctl.st[p].done);
  const Acc* kc = reinterpret_cast<const Acc*>(reinterpret_cast<const LsqrCoef<Acc>*>(ctl.coef) + p);
  h.K.inv_alpha = __ldcg(kc + 0);
  h.K.ab = __ldcg(kc + 1);
  h.K.phr = __ldcg(kc + 2);
  h.K.thr = __ldcg(kc + 3);
  h.K.inv_beta = __ldcg(kc + 4);
  h.K.ba = __ldcg(kc + 5);
  return h;
}

// Returns false (nothing written) when the problem has already stopped.
template <typename T, typename Acc>
__device__ int lsqr_pass_F(const LsqrProb<T, Acc>& P, const LsqrCtl& ctl, int p, bool init, bool first,
                           int r0, int c0, Acc* sm, Sums3<Acc>& red, Acc* cbr, Acc* cbc, int ph, bool wait_rel) {
  const int m = P.m;
  const TileGeom g = tile_geom(P.op, false);
  Acc* sx = sm;
  Acc* sz = sx + g.H * g.H;
  Acc* sbr = sz + g.H * TM;
  Acc* sbc = sbr + TM * band_pitch(g.w);
  using X = typename Traits<T>::X;
  const bool src = init ? (P.x0 != nullptr) : true;   // input vector: x0 (phase 0) or v
  const bool wtd = (P.solver == 0);
  Acc pu[PIX], px[PIX], py[PIX], pw_[PIX], pd[PIX], wx[PIX], wy[PIX];
  {
    const int rr = r0 + threadIdx.x;
#pragma unroll
    for (int j = 0; j < PIX; ++j) {
      const int cc = c0 + pix_col(j);
      pu[j] = px[j] = py[j] = pw_[j] = pd[j] = Acc(0);
      wx[j] = wy[j] = Acc(1);
      if (rr < m && cc < m) {
        const size_t i = rr + (size_t)cc * m;
        if (!init) {
          pu[j] = ldcg<T>(P.uA + i);
          px[j] = ldcg<T>(P.uLx + i);
          py[j] = ldcg<T>(P.uLy + i);
          if (!first) { pw_[j] = ldcg<T>(P.w + i); pd[j] = ldcg<X>(P.dlt + i); }
        }
        if (wtd) { wx[j] = to_acc(P.a0x[i]); wy[j] = to_acc(P.a0y[i]); }
      }
    }
  }
  const bool taps = P.op.ntaps > 0;
  if (src) {
    if (init) gather_tile<true, X, Acc>(P.x0, m, r0, c0, g, Acc(1), sx, taps);
    else gather_tile<true, T, Acc>(P.v, m, r0, c0, g, Acc(1), sx, taps);
    if (taps) load_taps<Acc>(P.op, sbr, reinterpret_cast<int*>(sbc));
    else if (!cbr) load_bands<Acc>(P.op, false, 0, r0, c0, g, sbr, sbc);
  }
  Acc Av[PIX] = {};
  if (src) tile_conv<Acc>(P.op, false, r0, c0, g, sx, sz, cbr ? cbr : sbr, cbc ? cbc : sbc, Av, true);
  // the convolution needs the new vectors only; the coefficients and the
  // stop flag come from the previous phase's scalar update
  if (wait_rel) {
    const int d = lsqr_wait_release(ctl, ph);
    if (d != 0) return d > 0 ? -1 : -2;
  }
  const TileHead<Acc> h = load_head<Acc>(ctl, p);
  if (h.done) return 0;
  const Acc sc = init ? Acc(1) : h.K.inv_alpha;   // v = v~ / alpha
  const Acc sg = P.sg;
  const Acc ab = init ? Acc(0) : h.K.ab;
  const Acc phr = h.K.phr, thr = h.K.thr;
  const int r = r0 + threadIdx.x;
  const int lr = threadIdx.x - g.lo;
#pragma unroll
  for (int j = 0; j < PIX; ++j) {
    const int cl = pix_col(j);
    const int c = c0 + cl;
    if (r >= m || c >= m) continue;
    const size_t i = r + (size_t)c * m;
    const int lc = cl - g.lo;
    Acc v0 = 0, qx = 0, qy = 0;
    if (src) {
      const Acc x0 = sx[lc * g.H + lr];
      v0 = sc * x0;
      if (r < m - 1) qx = sc * (sx[lc * g.H + lr + 1] - x0);
      if (c < m - 1) qy = sc * (sx[(lc + 1) * g.H + lr] - x0);
    }
    qx *= wx[j];
    qy *= wy[j];
    const Acc av = sc * Av[j];
    Acc ua, ux, uy;
    if (init) {
      Acc cx = 0, cy = 0;
      if (P.solver == 1) { cx = to_acc(P.a0x[i]); cy = to_acc(P.a0y[i]); }
      else if (P.solver == 2) { cx = to_acc(P.a0x[i]) - to_acc(P.a1x[i]); cy = to_acc(P.a0y[i]) - to_acc(P.a1y[i]); }
      ua = to_acc(P.b[i]) - av;
      ux = sg * (cx - qx);
      uy = sg * (cy - qy);
      P.dlt[i] = store_cast<X, Acc>(Acc(0));
    } else {
      ua = av - ab * pu[j];
      ux = sg * qx - ab * px[j];
      uy = sg * qy - ab * py[j];
      if (first) {
        P.w[i] = store_cast<T, Acc>(v0);
      } else {
        const Acc wo = pw_[j];
        const Acc dn = pd[j] + phr * wo;
        P.dlt[i] = store_cast<X, Acc>(dn);
        P.w[i] = store_cast<T, Acc>(v0 - thr * wo);
        red.sq(1, dn);
        red.sq(2, wo);
      }
    }
    if (r == m - 1) ux = 0;
    if (c == m - 1) uy = 0;
    P.uA[i] = store_cast<T, Acc>(ua);
    P.uLx[i] = store_cast<T, Acc>(ux);
    P.uLy[i] = store_cast<T, Acc>(uy);
    red.sq(0, ua);
    red.sq(0, ux);
    red.sq(0, uy);
  }
  return 1;
}

template <typename T, typename Acc>
__device__ int lsqr_pass_B(const LsqrProb<T, Acc>& P, const LsqrCtl& ctl, int p, bool init,
                           int r0, int c0, Acc* sm, Sums3<Acc>& red, Acc* cbr, Acc* cbc, int ph, bool wait_rel) {
  const int m = P.m;
  const TileGeom g = tile_geom(P.op, true);
  Acc* sx = sm;
  Acc* sz = sx + g.H * g.H;
  Acc* sbr = sz + g.H * TM;
  Acc* sbc = sbr + TM * band_pitch(g.w);
  const bool wtd = (P.solver == 0);
  // L^T applied to the (unscaled) gradient planes of this thread's pixels, and the old v
  Acc lt[PIX], vo[PIX];
  {
    const int rr = r0 + threadIdx.x;
#pragma unroll
    for (int j = 0; j < PIX; ++j) {
      const int cc = c0 + pix_col(j);
      Acc l = 0, v = 0;
      if (rr < m && cc < m) {
        // all loads issued unconditionally (clamped neighbours), then combined
        const size_t i = rr + (size_t)cc * m;
        const bool dn = rr < m - 1, up = rr > 0, rt = cc < m - 1, lf = cc > 0;
        const size_t iu = up ? i - 1 : i, il = lf ? i - m : i;
        const Acc x0 = ldcg<T>(P.uLx + i), x1 = ldcg<T>(P.uLx + iu);
        const Acc y0 = ldcg<T>(P.uLy + i), y1 = ldcg<T>(P.uLy + il);
        Acc wx0 = 1, wx1 = 1, wy0 = 1, wy1 = 1;
        if (wtd) { wx0 = to_acc(P.a0x[i]); wx1 = to_acc(P.a0x[iu]); wy0 = to_acc(P.a0y[i]); wy1 = to_acc(P.a0y[il]); }
        if (!init) v = ldcg<T>(P.v + i);
        if (dn) l -= x0 * wx0;
        if (up) l += x1 * wx1;
        if (rt) l -= y0 * wy0;
        if (lf) l += y1 * wy1;
      }
      lt[j] = l;
      vo[j] = v;
    }
  }
  const bool taps = P.op.ntaps > 0;
  gather_tile<true, T, Acc>(P.uA, m, r0, c0, g, Acc(1), sx, taps);
  if (taps) load_taps<Acc>(P.op, sbr, reinterpret_cast<int*>(sbc));
  else if (!cbr) load_bands<Acc>(P.op, true, 0, r0, c0, g, sbr, sbc);
  Acc At[PIX] = {};
  tile_conv<Acc>(P.op, true, r0, c0, g, sx, sz, cbr ? cbr : sbr, cbc ? cbc : sbc, At, true);
  if (wait_rel) {
    const int d = lsqr_wait_release(ctl, ph);
    if (d != 0) return d > 0 ? -1 : -2;
  }
  const TileHead<Acc> h = load_head<Acc>(ctl, p);
  if (h.done) return 0;
  const Acc ib = h.K.inv_beta;                    // u = u~ / beta
  const Acc sgb = P.sg * ib;
  const Acc ba = init ? Acc(0) : h.K.ba;
  const int r = r0 + threadIdx.x;
#pragma unroll
  for (int j = 0; j < PIX; ++j) {
    const int c = c0 + pix_col(j);
    if (r >= m || c >= m) continue;
    const size_t i = r + (size_t)c * m;
    Acc vt = ib * At[j] + sgb * lt[j];
    if (!init) vt -= ba * vo[j];
    P.v[i] = store_cast<T, Acc>(vt);
    red.sq(0, vt);
  }
  return 1;
}

// ---- direct level-0 path (op.toep, float working precision) ---------------
// The same two passes over a tile in the vector mapping of toep.cuh. All of
// a tile's inputs arrive by asynchronous copies on one mbarrier: the halo
// window by one TMA box copy (thread 0) and the pointwise operands by bulk
// copies into staging slots (warp y fills slot y, one column per lane), so
// no operand occupies registers while the convolution runs. Every warp
// arrives once per tile (the barrier counts TY arrivals), announcing the
// bytes it copies. The copies follow the barrier at the top of the tile
// (the previous tile's reads of the buffers are done) and the grid barrier
// that published the vectors; a proxy fence orders them after both.

// Warp-level: announce and issue the copy of one vector (p, elements of esz
// bytes; null: none) of tile (r0, c0) into `slot` (column c0 + j at slot
// column j + 1; with `left`, column c0 - 1 at slot column 0 when c0 > 0).
// `extra`: bytes of further copies this warp's lane 0 issues afterwards.
__device__ __forceinline__ void toep_stage(unsigned char* slot, const void* p, int esz, bool left, int r0, int c0,
                                           int m, uint64_t* bar, unsigned extra) {
  const int lane = threadIdx.x;
  const unsigned colb = (unsigned)(TM * esz);
  const bool lft = p && left && c0 > 0;
  if (lane == 0) {
    fence_proxy_async();
    mbar_arrive_expect_tx(bar, extra + (p ? colb * (32u + (lft ? 1u : 0u)) : 0u));
  }
  __syncwarp();
  if (p) {
    fence_proxy_async();
    const char* base = static_cast<const char*>(p) + (size_t)r0 * esz;
    bulk_load(slot + (lane + 1) * colb, base + (size_t)(c0 + lane) * m * esz, colb, bar);
    if (lane == 0 && lft) bulk_load(slot, base + (size_t)(c0 - 1) * m * esz, colb, bar);
  }
}

// Warp-level (the warp without a slot): announce and issue the copy of the
// taps of the level (2 * nterms * w floats, rounded up to 16 bytes; the
// arena allocation behind them is 256-byte granular) into `dst`.
__device__ __forceinline__ void toep_stage_taps(float* dst, const BandOp<float>& op, uint64_t* bar) {
  if (threadIdx.x == 0) {
    const unsigned bytes = (unsigned)((2 * op.nterms * op.w * 4 + 15) & ~15);
    fence_proxy_async();
    mbar_arrive_expect_tx(bar, bytes);
    bulk_load(dst, op.tp, bytes, bar);
  }
  __syncwarp();
}

// Waits for the tile's copies (every thread). A copy from L2/HBM lands within
// microseconds; the wait gives up after TOEP_COPY_LIMIT_NS, flags the error
// for the whole grid and waits once more, also bounded, for copies still in
// flight. Returns false (uniform over the block) on expiry.
constexpr unsigned long long TOEP_COPY_LIMIT_NS = 1000000000ull;
__device__ __forceinline__ bool toep_wait(const LsqrCtl& ctl, uint64_t* bar, unsigned& par) {
  const bool ok = mbar_wait_bounded(bar, par, TOEP_COPY_LIMIT_NS);
  if (__syncthreads_or(!ok)) {
    if (threadIdx.x == 0 && threadIdx.y == 0) {
      atomicExch(&ctl.gb->error, 1);
      mbar_wait_bounded(bar, par, TOEP_COPY_LIMIT_NS);
    }
    __syncthreads();
    return false;
  }
  par ^= 1u;
  return true;
}

// 4 values of this thread's pixels (rows 4a.., slot column cl + 1 + dc)
template <typename E>
__device__ __forceinline__ void slot4(const unsigned char* slot, int a, int cl, int dc, float (&o)[4]) {
  ld4s(reinterpret_cast<const E*>(slot) + (cl + 1 + dc) * TM + 4 * a, o);
}

template <typename T>
__device__ int lsqr_pass_F_toep(const LsqrProb<T, float>& P, const LsqrCtl& ctl, int p, bool init, bool first,
                                int r0, int c0, unsigned char* win, float* sz, unsigned char* slots,
                                Sums3<float>& red, int ph, bool wait_rel, uint64_t* bar, unsigned& par) {
  using X = typename Traits<T>::X;
  const int m = P.m;
  const BandOp<float>& op = P.op;
  const ToepGeom g = toep_geom(op.dlo, op.w);
  const bool src = init ? (P.x0 != nullptr) : true;   // input vector: x0 (phase 0) or v
  const bool wtd = (P.solver == 0);
  const int tid = threadIdx.x + 32 * threadIdx.y;
  const int a = tid & 7, cl = tid >> 3;
  const int r = r0 + 4 * a, c = c0 + cl;
  const size_t i = r + (size_t)c * m;
  float* stp = reinterpret_cast<float*>(slots + TOEP_SLOTS * TOEP_SLOT_BYTES);
  // slots: 0 u~_A | b, 1 u~_Lx | a1x, 2 u~_Ly | a1y, 3 w, 4 delta, 5 a0x, 6 a0y
  {
    const void* sp = nullptr;
    int esz = (int)sizeof(T);
    switch (threadIdx.y) {
      case 0: sp = init ? (const void*)P.b : (const void*)P.uA; break;
      case 1: sp = init ? (P.solver == 2 ? (const void*)P.a1x : nullptr) : (const void*)P.uLx; break;
      case 2: sp = init ? (P.solver == 2 ? (const void*)P.a1y : nullptr) : (const void*)P.uLy; break;
      case 3: sp = (!init && !first) ? (const void*)P.w : nullptr; break;
      case 4: sp = (!init && !first) ? (const void*)P.dlt : nullptr; esz = (int)sizeof(X); break;
      case 5: sp = (wtd || init) ? (const void*)P.a0x : nullptr; break;
      case 6: sp = (wtd || init) ? (const void*)P.a0y : nullptr; break;
      default: break;
    }
    const int wesz = init ? (int)sizeof(X) : (int)sizeof(T);
    const unsigned wbytes = (src && threadIdx.y == 0) ? (unsigned)(g.RB * g.CB * wesz) : 0u;
    if (threadIdx.y == TOEP_SLOTS) toep_stage_taps(stp, op, bar);
    else toep_stage(slots + threadIdx.y * TOEP_SLOT_BYTES, sp, esz, false, r0, c0, m, bar, wbytes);
    if (src && tid == 0) tma_load_2d(win, init ? P.tm_x0 : P.tm_v, r0 + g.f8, c0 + op.dlo, bar);
  }
  if (!toep_wait(ctl, bar, par)) return -2;
  // the input at this thread's pixels and their lower / right neighbours
  float x0v[4] = {0.f, 0.f, 0.f, 0.f}, xdn[4] = {0.f, 0.f, 0.f, 0.f}, xrt[4] = {0.f, 0.f, 0.f, 0.f};
  float Av[4] = {0.f, 0.f, 0.f, 0.f};
  if (src) {
    const int wr = 4 * a - g.f8, wc = cl - op.dlo;
    if (init) {
      const X* sx = reinterpret_cast<const X*>(win);
      toep_conv_any<X>(g, op.w, op.nterms, stp, false, sx, sz, Av);
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        x0v[j] = win_val(sx, wc * g.RB + wr + j);
        xdn[j] = win_val(sx, wc * g.RB + wr + j + 1);
        xrt[j] = win_val(sx, (wc + 1) * g.RB + wr + j);
      }
    } else {
      const T* sx = reinterpret_cast<const T*>(win);
      toep_conv_any<T>(g, op.w, op.nterms, stp, false, sx, sz, Av);
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        x0v[j] = win_val(sx, wc * g.RB + wr + j);
        xdn[j] = win_val(sx, wc * g.RB + wr + j + 1);
        xrt[j] = win_val(sx, (wc + 1) * g.RB + wr + j);
      }
    }
  }
  if (wait_rel) {
    const int d = lsqr_wait_release(ctl, ph);
    if (d != 0) return d > 0 ? -1 : -2;
  }
  const TileHead<float> h = load_head<float>(ctl, p);
  if (h.done) return 0;
  const float sc = init ? 1.f : h.K.inv_alpha;   // v = v~ / alpha
  const float sg = P.sg;
  const float ab = init ? 0.f : h.K.ab;
  const float phr = h.K.phr, thr = h.K.thr;
  float wx[4] = {1.f, 1.f, 1.f, 1.f}, wy[4] = {1.f, 1.f, 1.f, 1.f};
  if (wtd) {
    slot4<T>(slots + 5 * TOEP_SLOT_BYTES, a, cl, 0, wx);
    slot4<T>(slots + 6 * TOEP_SLOT_BYTES, a, cl, 0, wy);
  }
  float oA[4], oX[4], oY[4], oW[4], oD[4];
  if (init) {
    float bb[4], cx[4] = {0.f, 0.f, 0.f, 0.f}, cy[4] = {0.f, 0.f, 0.f, 0.f};
    slot4<T>(slots, a, cl, 0, bb);
    if (P.solver == 1 || P.solver == 2) {
      slot4<T>(slots + 5 * TOEP_SLOT_BYTES, a, cl, 0, cx);
      slot4<T>(slots + 6 * TOEP_SLOT_BYTES, a, cl, 0, cy);
    }
    if (P.solver == 2) {
      float ex[4], ey[4];
      slot4<T>(slots + 1 * TOEP_SLOT_BYTES, a, cl, 0, ex);
      slot4<T>(slots + 2 * TOEP_SLOT_BYTES, a, cl, 0, ey);
#pragma unroll
      for (int j = 0; j < 4; ++j) { cx[j] -= ex[j]; cy[j] -= ey[j]; }
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int rj = r + j;
      float qx = 0.f, qy = 0.f;
      if (src) {
        if (rj < m - 1) qx = xdn[j] - x0v[j];
        if (c < m - 1) qy = xrt[j] - x0v[j];
      }
      qx *= wx[j];
      qy *= wy[j];
      const float ua = bb[j] - Av[j];
      float ux = sg * (cx[j] - qx);
      float uy = sg * (cy[j] - qy);
      oD[j] = 0.f;
      if (rj == m - 1) ux = 0.f;
      if (c == m - 1) uy = 0.f;
      oA[j] = ua; oX[j] = ux; oY[j] = uy;
      red.sq(0, ua);
      red.sq(0, ux);
      red.sq(0, uy);
    }
    st4(P.dlt + i, oD);
  } else {
    float pu[4], px[4], py[4], pw_[4] = {0.f, 0.f, 0.f, 0.f}, pd[4] = {0.f, 0.f, 0.f, 0.f};
    slot4<T>(slots, a, cl, 0, pu);
    slot4<T>(slots + 1 * TOEP_SLOT_BYTES, a, cl, 0, px);
    slot4<T>(slots + 2 * TOEP_SLOT_BYTES, a, cl, 0, py);
    if (!first) {
      slot4<T>(slots + 3 * TOEP_SLOT_BYTES, a, cl, 0, pw_);
      slot4<X>(slots + 4 * TOEP_SLOT_BYTES, a, cl, 0, pd);
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int rj = r + j;
      const float v0 = sc * x0v[j];
      float qx = 0.f, qy = 0.f;
      if (rj < m - 1) qx = sc * (xdn[j] - x0v[j]);
      if (c < m - 1) qy = sc * (xrt[j] - x0v[j]);
      qx *= wx[j];
      qy *= wy[j];
      const float av = sc * Av[j];
      const float ua = av - ab * pu[j];
      float ux = sg * qx - ab * px[j];
      float uy = sg * qy - ab * py[j];
      if (first) {
        oW[j] = v0;
      } else {
        const float wo = pw_[j];
        const float dn = pd[j] + phr * wo;
        oD[j] = dn;
        oW[j] = v0 - thr * wo;
        red.sq(1, dn);
        red.sq(2, wo);
      }
      if (rj == m - 1) ux = 0.f;
      if (c == m - 1) uy = 0.f;
      oA[j] = ua; oX[j] = ux; oY[j] = uy;
      red.sq(0, ua);
      red.sq(0, ux);
      red.sq(0, uy);
    }
    st4(P.w + i, oW);
    if (!first) st4(P.dlt + i, oD);
  }
  st4(P.uA + i, oA);
  st4(P.uLx + i, oX);
  st4(P.uLy + i, oY);
  return 1;
}

template <typename T>
__device__ int lsqr_pass_B_toep(const LsqrProb<T, float>& P, const LsqrCtl& ctl, int p, bool init, int r0, int c0,
                                unsigned char* win, float* sz, unsigned char* slots, Sums3<float>& red, int ph,
                                bool wait_rel, uint64_t* bar, unsigned& par) {
  const int m = P.m;
  const BandOp<float>& op = P.op;
  const ToepGeom g = toep_geom(op.dlo, op.w);
  const bool wtd = (P.solver == 0);
  const int tid = threadIdx.x + 32 * threadIdx.y;
  const int a = tid & 7, cl = tid >> 3;
  const int r = r0 + 4 * a, c = c0 + cl;
  const size_t i = r + (size_t)c * m;
  float* stp = reinterpret_cast<float*>(slots + TOEP_SLOTS * TOEP_SLOT_BYTES);
  // slots: 0 u~_Lx, 1 u~_Ly (with column c0 - 1), 2 v~, 5 a0x, 6 a0y (with column c0 - 1)
  {
    const void* sp = nullptr;
    bool left = false;
    switch (threadIdx.y) {
      case 0: sp = P.uLx; break;
      case 1: sp = P.uLy; left = true; break;
      case 2: sp = init ? nullptr : (const void*)P.v; break;
      case 5: sp = wtd ? (const void*)P.a0x : nullptr; break;
      case 6: sp = wtd ? (const void*)P.a0y : nullptr; left = true; break;
      default: break;
    }
    const unsigned wbytes = threadIdx.y == 0 ? (unsigned)(g.RB * g.CB * (int)sizeof(T)) : 0u;
    if (threadIdx.y == TOEP_SLOTS) toep_stage_taps(stp, op, bar);
    else toep_stage(slots + threadIdx.y * TOEP_SLOT_BYTES, sp, (int)sizeof(T), left, r0, c0, m, bar, wbytes);
    if (tid == 0) tma_load_2d(win, P.tm_u, r0 + g.f8, c0 + op.dlo, bar);
  }
  // the row above the tile (first pixel of the threads with a = 0; the
  // others find it in the staged column)
  float xm1 = 0.f, wxm1 = 1.f;
  if (r > 0 && a == 0) {
    xm1 = ldcg<T>(P.uLx + i - 1);
    if (wtd) wxm1 = to_acc(P.a0x[i - 1]);
  }
  if (!toep_wait(ctl, bar, par)) return -2;
  float At[4] = {0.f, 0.f, 0.f, 0.f};
  toep_conv_any<T>(g, op.w, op.nterms, stp, true, reinterpret_cast<const T*>(win), sz, At);
  if (wait_rel) {
    const int d = lsqr_wait_release(ctl, ph);
    if (d != 0) return d > 0 ? -1 : -2;
  }
  const TileHead<float> h = load_head<float>(ctl, p);
  if (h.done) return 0;
  // L^T applied to the (unscaled) gradient planes at this thread's pixels:
  // the row above comes from the thread's own column except for its first
  // pixel, the column to the left from the staged column c - 1
  float x4[4], y4[4], yl[4] = {0.f, 0.f, 0.f, 0.f}, vo[4] = {0.f, 0.f, 0.f, 0.f};
  float wx4[4] = {1.f, 1.f, 1.f, 1.f}, wy4[4] = {1.f, 1.f, 1.f, 1.f}, wyl[4] = {1.f, 1.f, 1.f, 1.f};
  slot4<T>(slots, a, cl, 0, x4);
  if (a > 0) {
    xm1 = win_val(reinterpret_cast<const T*>(slots), (cl + 1) * TM + 4 * a - 1);
    if (wtd) wxm1 = win_val(reinterpret_cast<const T*>(slots + 5 * TOEP_SLOT_BYTES), (cl + 1) * TM + 4 * a - 1);
  }
  slot4<T>(slots + 1 * TOEP_SLOT_BYTES, a, cl, 0, y4);
  if (c > 0) slot4<T>(slots + 1 * TOEP_SLOT_BYTES, a, cl, -1, yl);
  if (!init) slot4<T>(slots + 2 * TOEP_SLOT_BYTES, a, cl, 0, vo);
  if (wtd) {
    slot4<T>(slots + 5 * TOEP_SLOT_BYTES, a, cl, 0, wx4);
    slot4<T>(slots + 6 * TOEP_SLOT_BYTES, a, cl, 0, wy4);
    if (c > 0) slot4<T>(slots + 6 * TOEP_SLOT_BYTES, a, cl, -1, wyl);
  }
  const float ib = h.K.inv_beta;                    // u = u~ / beta
  const float sgb = P.sg * ib;
  const float ba = init ? 0.f : h.K.ba;
  float ov[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int rj = r + j;
    const float x1 = j ? x4[j - 1] : xm1, wx1 = j ? wx4[j - 1] : wxm1;
    float l = 0.f;
    if (rj < m - 1) l -= x4[j] * wx4[j];
    if (rj > 0) l += x1 * wx1;
    if (c < m - 1) l -= y4[j] * wy4[j];
    if (c > 0) l += yl[j] * wyl[j];
    float vt = ib * At[j] + sgb * l;
    if (!init) vt -= ba * vo[j];
    ov[j] = vt;
    red.sq(0, vt);
  }
  st4(P.v + i, ov);
  return 1;
}

// Scalar work once every tile of a problem has reported (run by one thread).
// Norms come from one rsqrt each (value = x * rsqrt(x)); the stopping tests
// compare squares, so no square root or divide is needed for them:
//   S1  rnorm <= btol*bnorm + atol*anorm*xnorm
//   S2  arnorm <= atol*anorm*rnorm          (anorm, rnorm > 0)
//   S3  anorm*||D_k||_F >= conlim
template <typename Acc>
__device__ __forceinline__ int lsqr_finish_F(const LsqrCtl& ctl, LsqrState S, LsqrState* st, LsqrCoef<Acc>* K,
                                             bool init, int it, const double (&tot)[3]) {
  const double ib = tot[0] > 0.0 ? rsqrt(tot[0]) : 0.0;
  const double beta_new = tot[0] * ib;
  if (init) {
    S.beta = beta_new;
    S.bnorm = beta_new;
    S.phibar = beta_new;
    S.it = 0;
    S.its = 0;
    if (beta_new == 0.0) { S.done = 1; S.stop = 5; }
  } else {
    if (it >= 2) {
      const int k = it - 1;           // iteration being tested
      S.dnorm2 += tot[2] * (S.irho_last * S.irho_last);
      const double xnorm2 = tot[1];
      const double rnorm = S.t_rnorm, arnorm = S.t_arnorm;
      const double lhs = rnorm - ctl.btol * S.bnorm;
      int stop = 0;
      if (lhs <= 0.0 || lhs * lhs <= ctl.atol * ctl.atol * S.anorm2 * xnorm2) stop = 1;
      else if (S.anorm2 > 0.0 && rnorm > 0.0 && arnorm * arnorm <= ctl.atol * ctl.atol * S.anorm2 * rnorm * rnorm) stop = 2;
      else if (S.anorm2 * S.dnorm2 >= ctl.conlim * ctl.conlim) stop = 3;
      else if (k >= ctl.maxit) stop = 4;
      if (stop) { S.done = 1; S.stop = stop; S.its = k; }
    }
    S.beta = beta_new;
    S.it = it;
  }
  *st = S;
  // coefficients of pass B: u = u~ / beta_{i+1}, v~ -= (beta_{i+1} / alpha_i) v~
  K->inv_beta = (Acc)ib;
  K->ba = (!init && S.alpha > 0.0) ? (Acc)(beta_new * (double)K->inv_alpha) : Acc(0);
  return S.done;
}

template <typename Acc>
__device__ __forceinline__ int lsqr_finish_B(LsqrState S, LsqrState* st, LsqrCoef<Acc>* K, bool init,
                                             const double (&tot)[3]) {
  const double ia = tot[0] > 0.0 ? rsqrt(tot[0]) : 0.0;
  const double alpha_new = tot[0] * ia;
  if (init) {
    S.alpha = alpha_new;
    S.rhobar = alpha_new;
    S.anorm2 = 0.0;
    S.dnorm2 = 0.0;
    S.phi_rho = 0.0;
    S.theta_rho = 0.0;
    if (alpha_new == 0.0) { S.done = 1; S.stop = 5; S.its = 0; }
  } else {
    const double alpha = S.alpha, beta = S.beta;
    S.anorm2 += alpha * alpha + beta * beta;
    const double rho2 = S.rhobar * S.rhobar + beta * beta;
    const double irho = rsqrt(rho2);        // one rsqrt gives 1/rho
    const double c = S.rhobar * irho, s = beta * irho;
    const double theta = s * alpha_new;
    S.rhobar = -c * alpha_new;
    const double phi = c * S.phibar;
    S.phibar = s * S.phibar;
    S.phi_rho = phi * irho;
    S.theta_rho = theta * irho;
    S.irho_last = irho;
    S.t_rnorm = S.phibar;
    S.t_arnorm = S.phibar * alpha_new * fabs(c);
    S.alpha = alpha_new;
  }
  *st = S;
  // coefficients of the next pass F
  K->inv_alpha = (Acc)ia;
  K->ab = S.beta > 0.0 ? (Acc)(S.alpha * (double)K->inv_beta) : Acc(0);
  K->phr = (Acc)S.phi_rho;
  K->thr = (Acc)S.theta_rho;
  return S.done;
}

// Per-tile partial of the three sums into part[tile*3 .. tile*3+2] (24 bytes).
// Float working precision: TwoSum butterflies within the warps and across
// them, stored as (hi, lo) float pairs -- no FP64 instruction, whose issue
// costs ~64 cycles per warp instruction on this part. Double working
// precision: FP64 block sum, stored as doubles.
__device__ __forceinline__ void tile_partial(const Sums3<float>& red, double* part_tile, double* scratch) {
  const int tid = threadIdx.x + 32 * threadIdx.y, lane = tid & 31, wid = tid >> 5;
  float2* sw = reinterpret_cast<float2*>(scratch);          // [3][8]
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const float2 r = warp_df_pair(red.h[k], red.l[k]);
    if (lane == 0) sw[k * 8 + wid] = r;
  }
  __syncthreads();
  if (wid == 0) {
    float2* out = reinterpret_cast<float2*>(part_tile);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      float h = lane < TY ? sw[k * 8 + lane].x : 0.f, l = lane < TY ? sw[k * 8 + lane].y : 0.f;
#pragma unroll
      for (int o = 4; o > 0; o >>= 1) {
        const float h2 = __shfl_xor_sync(0xffffffffu, h, o), l2 = __shfl_xor_sync(0xffffffffu, l, o);
        df_add(h, l, h2, l2);
      }
      if (lane == 0) out[k] = make_float2(h, l);
    }
  }
}
__device__ __forceinline__ void tile_partial(const Sums3<double>& red, double* part_tile, double* scratch) {
  double tot[3];
  block_sum_to0<3, double>(red.h, tot, scratch);
  if (threadIdx.x == 0 && threadIdx.y == 0) {
#pragma unroll
    for (int k = 0; k < 3; ++k) part_tile[k] = tot[k];
  }
}

// Sum of a problem's tile partials by one warp, in tile order; result in lane 0.
template <typename Acc>
__device__ __forceinline__ void problem_partials(const double* part, int ntiles, double (&tot)[3]);
template <>
__device__ __forceinline__ void problem_partials<float>(const double* part, int ntiles, double (&tot)[3]) {
  constexpr int PB = 8;
  const int lane = threadIdx.x;
  const float2* pp = reinterpret_cast<const float2*>(part);
  float h[3] = {0.f, 0.f, 0.f}, l[3] = {0.f, 0.f, 0.f};
  for (int t0 = lane; t0 < ntiles; t0 += 32 * PB) {
    float2 q[PB][3];
#pragma unroll
    for (int b = 0; b < PB; ++b) {
      const int t = t0 + 32 * b;
#pragma unroll
      for (int k = 0; k < 3; ++k) q[b][k] = t < ntiles ? __ldcg(pp + (size_t)t * 3 + k) : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int b = 0; b < PB; ++b)
#pragma unroll
      for (int k = 0; k < 3; ++k) df_add(h[k], l[k], q[b][k].x, q[b][k].y);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1)
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const float h2 = __shfl_xor_sync(0xffffffffu, h[k], o), l2 = __shfl_xor_sync(0xffffffffu, l[k], o);
      df_add(h[k], l[k], h2, l2);
    }
#pragma unroll
  for (int k = 0; k < 3; ++k) tot[k] = (double)h[k] + (double)l[k];
}
template <>
__device__ __forceinline__ void problem_partials<double>(const double* part, int ntiles, double (&tot)[3]) {
  constexpr int PB = 8;
  const int lane = threadIdx.x;
  tot[0] = tot[1] = tot[2] = 0.0;
  for (int t0 = lane; t0 < ntiles; t0 += 32 * PB) {
    double q[PB][3];
#pragma unroll
    for (int b = 0; b < PB; ++b) {
      const int t = t0 + 32 * b;
#pragma unroll
      for (int k = 0; k < 3; ++k) q[b][k] = t < ntiles ? __ldcg(part + (size_t)t * 3 + k) : 0.0;
    }
#pragma unroll
    for (int b = 0; b < PB; ++b)
#pragma unroll
      for (int k = 0; k < 3; ++k) tot[k] += q[b][k];
  }
#pragma unroll
  for (int k = 0; k < 3; ++k) tot[k] = warp_sum(tot[k]);
}

// Tile partials of phase ph (0, 1, 2, ...): two buffers by phase parity,
// since blocks write the next phase's partials while the finishing block may
// still read this phase's.
__device__ __forceinline__ double* phase_part(const LsqrCtl& ctl, int ph) {
  return ctl.part + (size_t)(ph & 1) * ctl.ntiles * 3;
}

// End of phase ph, a barrier in two halves. Every block adds one to a
// counter that only grows. The block that brings it to G (ph + 1) reduces
// every problem's partials (warp w takes problems w, w + 8, ...; tile order),
// runs the scalar updates and publishes them with gen = ph + 1 and the
// all-stopped decision. Every other block waits only until all blocks have
// arrived: its next loads and convolution read the new vectors, not the new
// coefficients, and it meets the publication later (lsqr_wait_release).
// Returns -1 on timeout.
template <typename T, typename Acc>
__device__ int lsqr_phase_arrive(const LsqrProb<T, Acc>* probs, const LsqrCtl& ctl, LsqrCoef<Acc>* coef, bool isF,
                                 int it, int ph) {
  __shared__ int s_last, s_ok, s_live;
  GridBarrier* gb = ctl.gb;
  const int tid = threadIdx.x + 32 * threadIdx.y;
  const unsigned target = gridDim.x * (unsigned)(ph + 1);
  using aref = cuda::atomic_ref<unsigned, cuda::thread_scope_device>;
  __syncthreads();
  if (tid == 0) {
    s_ok = (*(volatile int*)&gb->error == 0);
    s_last = 0;
    s_live = 0;
    // release: this block's writes of the phase (ordered before by the block
    // barrier) become visible to whoever acquires the counter
    if (s_ok) s_last = (aref(gb->count).fetch_add(1u, cuda::memory_order_acq_rel) == target - 1);
  }
  __syncthreads();
  if (!s_ok) return -1;
  if (s_last) {
    const int warp = tid >> 5, lane = tid & 31;
    for (int p = warp; p < ctl.nprob; p += (32 * TY) / 32) {
      const LsqrProb<T, Acc>& P = probs[p];
      // state and tile partials requested together, partials summed in tile order
      LsqrState S;
      if (lane == 0) S = load_state(&ctl.st[p]);
      double tot[3];
      problem_partials<Acc>(phase_part(ctl, ph) + (size_t)P.tile_begin * 3, P.ntiles, tot);
      if (lane == 0 && !S.done) {
        const int done = isF ? lsqr_finish_F<Acc>(ctl, S, &ctl.st[p], coef + p, it == 0, it, tot)
                             : lsqr_finish_B<Acc>(S, &ctl.st[p], coef + p, it == 0, tot);
        if (!done) s_live = 1;
      }
    }
    __syncthreads();
    if (tid == 0) {
      gb->decision = s_live ? 0 : 1;
      // release: the scalar updates of this block become visible with gen
      aref(gb->gen).store((unsigned)(ph + 1), cuda::memory_order_release);
    }
  } else if (tid == 0) {
    const unsigned long long t0 = globaltimer_ns();
    unsigned spins = 0;
    while (aref(gb->count).load(cuda::memory_order_acquire) < target) {
      if (*(volatile int*)&gb->error) { s_ok = 0; break; }
      if (((++spins) & spin_mask(ctl)) == 0 && globaltimer_ns() - t0 > ctl.limit_ns) {
        atomicExch(&gb->error, 1);
        s_ok = 0;
        break;
      }
    }
  }
  __syncthreads();
  return s_ok ? 0 : -1;
}

// Wait for the scalars of phase ph - 1 (gen >= ph). Returns the decision
// (1: every problem has stopped), or -1 on timeout. Uniform over the block.
__device__ int lsqr_wait_release(const LsqrCtl& ctl, int ph) {
  __shared__ int s_res;
  if (ph == 0) return 0;
  using aref = cuda::atomic_ref<unsigned, cuda::thread_scope_device>;
  GridBarrier* gb = ctl.gb;
  if (threadIdx.x == 0 && threadIdx.y == 0) {
    const unsigned long long t0 = globaltimer_ns();
    unsigned spins = 0;
    int res = 0;
    while (aref(gb->gen).load(cuda::memory_order_acquire) < (unsigned)ph) {
      if (*(volatile int*)&gb->error) { res = -1; break; }
      if (((++spins) & spin_mask(ctl)) == 0 && globaltimer_ns() - t0 > ctl.limit_ns) {
        atomicExch(&gb->error, 1);
        res = -1;
        break;
      }
    }
    s_res = res < 0 ? -1 : *(volatile int*)&gb->decision;
  }
  __syncthreads();
  return s_res;
}

constexpr int LSQR_TCACHE = 4;   // tile descriptors a block keeps in shared memory

template <typename T, typename Acc>
__global__ void __launch_bounds__(256, 2) k_lsqr(const LsqrProb<T, Acc>* __restrict__ probs, LsqrCtl ctl) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Acc* sm = reinterpret_cast<Acc*>(smem_raw);
  // window of the direct level-0 path: the dynamic buffer rounded up to the
  // 128-byte alignment of a TMA destination (the host adds the slack)
  unsigned char* win = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 127) &
                                                        ~static_cast<uintptr_t>(127));
  __shared__ __align__(8) uint64_t s_bar;   // completion of the window copy
  unsigned par = 0;                         // parity of the next completion
  __shared__ double scratch[3 * 32];
  // raw storage: the descriptors are copied in word by word below (a
  // __shared__ object of the struct type would ask for a constructor)
  __shared__ __align__(16) unsigned char s_prob_raw[LSQR_TCACHE * sizeof(LsqrProb<T, Acc>)];
  LsqrProb<T, Acc>* s_prob = reinterpret_cast<LsqrProb<T, Acc>*>(s_prob_raw);
  __shared__ int s_pid[LSQR_TCACHE];
  __shared__ int s_skip[2];
  LsqrCoef<Acc>* coef = reinterpret_cast<LsqrCoef<Acc>*>(ctl.coef);
  const unsigned G = gridDim.x;
  const int tid = threadIdx.x + 32 * threadIdx.y;
  // the descriptors of this block's first tiles stay in shared memory for the
  // whole launch (the loads after a grid barrier then start from registers)
  for (int k = 0; k < LSQR_TCACHE; ++k) {
    const int tile = blockIdx.x + k * (int)G;
    if (tile >= ctl.ntiles) break;
    const int p = __ldg(ctl.tile_prob + tile);
    const int* src = reinterpret_cast<const int*>(probs + p);
    int* dst = reinterpret_cast<int*>(&s_prob[k]);
    for (int w = tid; w < (int)(sizeof(LsqrProb<T, Acc>) / sizeof(int)); w += 32 * TY) dst[w] = src[w];
    if (tid == 0) s_pid[k] = p;
  }
  if (tid == 0) mbar_init(&s_bar, TY);   // one arrival per warp and tile (direct path)
  __syncthreads();
  // band rows of the cached tiles, forward and transposed (one-term PSFs:
  // they are the same in every pass of the launch)
  if (ctl.band_cache) {
    for (int k = 0; k < LSQR_TCACHE; ++k) {
      const int tile = blockIdx.x + k * (int)G;
      if (tile >= ctl.ntiles) break;
      const LsqrProb<T, Acc>& P = s_prob[k];
      if (P.op.toep) continue;
      const int tl = tile - P.tile_begin;
      const int r0 = (tl % P.nt) * TM, c0 = (tl / P.nt) * TN;
      Acc* cb = sm + ctl.cache_off + (size_t)k * 4 * TM * ctl.band_pw;
      load_bands<Acc>(P.op, false, 0, r0, c0, tile_geom(P.op, false), cb, cb + TM * ctl.band_pw);
      load_bands<Acc>(P.op, true, 0, r0, c0, tile_geom(P.op, true), cb + 2 * TM * ctl.band_pw,
                      cb + 3 * TM * ctl.band_pw);
    }
    __syncthreads();
  }
  // phase 0: F(init), B(init); then F_i, B_i for i = 1, 2, ...; phase
  // ph = 2 i + half. The stop of every problem, decided with the scalars of
  // phase ph - 1, is read at the first tile of phase ph.
  for (int it = 0;; ++it) {
    for (int half = 0; half < 2; ++half) {
      const bool isF = (half == 0);
      const int ph = 2 * it + half;
      int k = 0;
      bool waited = false;   // this block has met the release of phase ph - 1
      for (int tile = blockIdx.x; tile < ctl.ntiles; tile += G, ++k) {
        const bool cached = k < LSQR_TCACHE;
        const int p = cached ? s_pid[k] : __ldg(ctl.tile_prob + tile);
        // tiles of a problem that has stopped are skipped before any load
        // (launches over several problems, which stop at different
        // iterations; a single problem ends the launch when it stops).
        // Thread 0 reads the flag for the whole block; it only ever goes from
        // 0 to 1, so a stale 0 costs one pass and nothing else.
        // (Two slots by tile parity: a thread can only write the slot of tile
        // k + 2 after every thread has passed the barrier of tile k + 1.)
        if (tid == 0) s_skip[k & 1] = (ph > 0 && ctl.nprob > 1) ? __ldcg(&ctl.st[p].done) : 0;
        __syncthreads();   // shared memory of the previous tile is free; s_skip is visible
        if (s_skip[k & 1]) continue;
        const LsqrProb<T, Acc>& P = cached ? s_prob[k] : probs[p];
        const int tl = tile - P.tile_begin;
        const int r0 = (tl % P.nt) * TM, c0 = (tl / P.nt) * TN;
        Sums3<Acc> red;
        Acc* cbr = nullptr;
        Acc* cbc = nullptr;
        if (cached && ctl.band_cache) {
          Acc* cb = sm + ctl.cache_off + (size_t)k * 4 * TM * ctl.band_pw + (isF ? 0 : 2 * TM * ctl.band_pw);
          cbr = cb;
          cbc = cb + TM * ctl.band_pw;
        }
        int rc;
        if constexpr (sizeof(Acc) == 4) {
          if (P.op.toep) {
            const ToepGeom tg = toep_geom(P.op.dlo, P.op.w);
            float* sz = reinterpret_cast<float*>(win + toep_win_bytes(tg));
            unsigned char* slots = win + toep_win_bytes(tg) + toep_z_bytes(tg);
            rc = isF ? lsqr_pass_F_toep<T>(P, ctl, p, it == 0, it == 1, r0, c0, win, sz, slots, red, ph, !waited,
                                           &s_bar, par)
                     : lsqr_pass_B_toep<T>(P, ctl, p, it == 0, r0, c0, win, sz, slots, red, ph, !waited, &s_bar, par);
          } else {
            rc = isF ? lsqr_pass_F<T, Acc>(P, ctl, p, it == 0, it == 1, r0, c0, sm, red, cbr, cbc, ph, !waited)
                     : lsqr_pass_B<T, Acc>(P, ctl, p, it == 0, r0, c0, sm, red, cbr, cbc, ph, !waited);
          }
        } else {
          rc = isF ? lsqr_pass_F<T, Acc>(P, ctl, p, it == 0, it == 1, r0, c0, sm, red, cbr, cbc, ph, !waited)
                   : lsqr_pass_B<T, Acc>(P, ctl, p, it == 0, r0, c0, sm, red, cbr, cbc, ph, !waited);
        }
        waited = true;
        if (rc < 0) return;    // every problem has stopped, or a wait timed out (uniform over the block)
        if (rc == 0) continue;
        tile_partial(red, phase_part(ctl, ph) + (size_t)tile * 3, scratch);
      }
      // a block whose tiles were all skipped still meets the release (it
      // carries the all-stopped decision) before it arrives
      if (!waited && lsqr_wait_release(ctl, ph) != 0) return;
      if (lsqr_phase_arrive<T, Acc>(probs, ctl, coef, isF, it, ph) < 0) return;
    }
  }
}

}  // namespace db
