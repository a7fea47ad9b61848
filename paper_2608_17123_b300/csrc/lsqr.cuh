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
#include "ops.cuh"

namespace db {

template <typename T, typename Acc>
struct LsqrProb {
  BandOp<Acc> op;
  int m, solver;                 // 0 IRLS (weighted D), 1 MM (c = a0), 2 SB (c = a0 - a1)
  double gamma;
  const T* b;
  const T* x0;                   // null: start from zero
  const T *a0x, *a0y, *a1x, *a1y;
  T *uA, *uLx, *uLy, *v, *w, *dlt;
  int tile_begin, ntiles, nt;    // tiles [tile_begin, tile_begin + ntiles), nt per side
};

struct LsqrState {
  double alpha, beta, rhobar, phibar, anorm2, dnorm2, bnorm;
  double phi_rho, theta_rho, rho_last, t_rnorm, t_arnorm;
  int it, done, its, stop;       // stop: 1 S1, 2 S2, 3 S3, 4 maxit, 5 zero rhs/A^T rhs
};

struct LsqrCtl {
  double atol, btol, conlim;
  int maxit, nprob, ntiles;
  const int* tile_prob;          // [ntiles] problem of each tile
  double* part;                  // [ntiles * 3] per-tile partial sums
  unsigned* cnt;                 // [nprob] tiles finished in the current phase
  LsqrState* st;                 // [nprob]
  GridBarrier* gb;
  unsigned long long limit_ns;
};

template <typename T> __device__ __forceinline__ typename Traits<T>::Acc ldcg(const T* p);
template <> __device__ __forceinline__ float ldcg<float>(const float* p) { return __ldcg(p); }
template <> __device__ __forceinline__ double ldcg<double>(const double* p) { return __ldcg(p); }
template <> __device__ __forceinline__ float ldcg<__nv_bfloat16>(const __nv_bfloat16* p) {
  unsigned short u = __ldcg(reinterpret_cast<const unsigned short*>(p));
  return __bfloat162float(__ushort_as_bfloat16(u));
}

// Same as load_tile but bypassing L1 (data written earlier in this launch).
template <typename T, typename Acc>
__device__ __forceinline__ void load_tile_cg(const T* X, int m, int r0, int c0, const TileGeom& g,
                                             Acc scale, Acc* sx) {
  const int tid = threadIdx.x + 32 * threadIdx.y;
  const int H = g.H;
  for (int idx = tid; idx < H * H; idx += 32 * TY) {
    int cc = idx / H, rr = idx - cc * H;
    int gr = wrap(r0 + g.lo + rr, m), gc = wrap(c0 + g.lo + cc, m);
    sx[idx] = (Acc)ldcg<T>(X + gr + (size_t)gc * m) * scale;
  }
}

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

// Reduce this tile's NV partials; returns true in the block that completed the
// last tile of problem p (and has to finish the problem's reduction).
template <int NV>
__device__ __forceinline__ bool finish_tile(double (&red)[NV], double* part, unsigned* cnt, int tile,
                                            int p, int ntiles_p, double* scratch, int* s_flag) {
  block_sum<NV>(red, scratch);
  if (threadIdx.x == 0 && threadIdx.y == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) part[(size_t)tile * NV + k] = red[k];
    __threadfence();
    unsigned old = atomicAdd(&cnt[p], 1u);
    *s_flag = (old == (unsigned)ntiles_p - 1);
    __threadfence();
  }
  __syncthreads();
  return *s_flag != 0;
}

// Fixed-order sum of a problem's tile partials by warp 0 (result in lane 0).
template <int NV>
__device__ __forceinline__ void problem_sum(const double* part, int tile_begin, int ntiles, double (&out)[NV]) {
  const int lane = threadIdx.x;
#pragma unroll
  for (int k = 0; k < NV; ++k) out[k] = 0.0;
  for (int t = lane; t < ntiles; t += 32) {
#pragma unroll
    for (int k = 0; k < NV; ++k) out[k] += __ldcg(part + (size_t)(tile_begin + t) * NV + k);
  }
#pragma unroll
  for (int k = 0; k < NV; ++k) out[k] = warp_sum(out[k]);
}

template <typename T, typename Acc>
__device__ void lsqr_pass_F(const LsqrProb<T, Acc>& P, const LsqrState& S, bool init, bool first,
                            int r0, int c0, Acc* sm, double (&red)[3]) {
  const int m = P.m;
  const TileGeom g = tile_geom(P.op, false);
  Acc* sx = sm;
  Acc* sz = sx + g.H * g.H;
  Acc* sbr = sz + g.H * TM;
  Acc* sbc = sbr + TM * band_pitch(g.w);
  const T* src = init ? P.x0 : P.v;
  const Acc inv_alpha = init ? Acc(1) : (S.alpha > 0.0 ? (Acc)(1.0 / S.alpha) : Acc(0));
  Acc Av[PIX] = {};
  __syncthreads();
  if (src) {
    load_tile_cg<T, Acc>(src, m, r0, c0, g, inv_alpha, sx);
    tile_conv<Acc>(P.op, false, r0, c0, g, sx, sz, sbr, sbc, Av);
  }
  const Acc sg = (Acc)sqrt(P.gamma);
  const Acc ab = (!init && S.beta > 0.0) ? (Acc)(S.alpha / S.beta) : Acc(0);
  const Acc phr = (Acc)S.phi_rho, thr = (Acc)S.theta_rho;
  const int r = r0 + threadIdx.x;
  const int lr = threadIdx.x - g.lo;
  Acc s_u = 0, s_d = 0, s_w = 0;
#pragma unroll
  for (int j = 0; j < PIX; ++j) {
    const int cl = threadIdx.y + TY * j;
    const int c = c0 + cl;
    if (r >= m || c >= m) continue;
    const size_t i = r + (size_t)c * m;
    const int lc = cl - g.lo;
    Acc v0 = 0, qx = 0, qy = 0;
    if (src) {
      v0 = sx[lc * g.H + lr];
      if (r < m - 1) qx = sx[lc * g.H + lr + 1] - v0;
      if (c < m - 1) qy = sx[(lc + 1) * g.H + lr] - v0;
    }
    if (P.solver == 0) { qx *= to_acc(P.a0x[i]); qy *= to_acc(P.a0y[i]); }
    Acc ua, ux, uy;
    if (init) {
      Acc cx = 0, cy = 0;
      if (P.solver == 1) { cx = to_acc(P.a0x[i]); cy = to_acc(P.a0y[i]); }
      else if (P.solver == 2) { cx = to_acc(P.a0x[i]) - to_acc(P.a1x[i]); cy = to_acc(P.a0y[i]) - to_acc(P.a1y[i]); }
      ua = to_acc(P.b[i]) - Av[j];
      ux = sg * (cx - qx);
      uy = sg * (cy - qy);
      P.dlt[i] = store_cast<T, Acc>(Acc(0));
    } else {
      ua = Av[j] - ab * ldcg<T>(P.uA + i);
      ux = sg * qx - ab * ldcg<T>(P.uLx + i);
      uy = sg * qy - ab * ldcg<T>(P.uLy + i);
      if (first) {
        P.w[i] = store_cast<T, Acc>(v0);
      } else {
        const Acc wo = ldcg<T>(P.w + i);
        const Acc dn = ldcg<T>(P.dlt + i) + phr * wo;
        P.dlt[i] = store_cast<T, Acc>(dn);
        P.w[i] = store_cast<T, Acc>(v0 - thr * wo);
        s_d += dn * dn;
        s_w += wo * wo;
      }
    }
    if (r == m - 1) ux = 0;
    if (c == m - 1) uy = 0;
    P.uA[i] = store_cast<T, Acc>(ua);
    P.uLx[i] = store_cast<T, Acc>(ux);
    P.uLy[i] = store_cast<T, Acc>(uy);
    s_u += ua * ua + ux * ux + uy * uy;
  }
  red[0] = (double)s_u;
  red[1] = (double)s_d;
  red[2] = (double)s_w;
}

template <typename T, typename Acc>
__device__ void lsqr_pass_B(const LsqrProb<T, Acc>& P, const LsqrState& S, bool init,
                            int r0, int c0, Acc* sm, double (&red)[3]) {
  const int m = P.m;
  const TileGeom g = tile_geom(P.op, true);
  Acc* sx = sm;
  Acc* sz = sx + g.H * g.H;
  Acc* sbr = sz + g.H * TM;
  Acc* sbc = sbr + TM * band_pitch(g.w);
  const Acc inv_beta = S.beta > 0.0 ? (Acc)(1.0 / S.beta) : Acc(0);
  Acc At[PIX] = {};
  __syncthreads();
  load_tile_cg<T, Acc>(P.uA, m, r0, c0, g, inv_beta, sx);
  tile_conv<Acc>(P.op, true, r0, c0, g, sx, sz, sbr, sbc, At);
  const Acc sg = (Acc)sqrt(P.gamma);
  const Acc ba = (!init && S.alpha > 0.0) ? (Acc)(S.beta / S.alpha) : Acc(0);
  const int r = r0 + threadIdx.x;
  Acc s_v = 0;
  const bool wtd = (P.solver == 0);
#pragma unroll
  for (int j = 0; j < PIX; ++j) {
    const int c = c0 + threadIdx.y + TY * j;
    if (r >= m || c >= m) continue;
    const size_t i = r + (size_t)c * m;
    Acc lt = 0;
    if (r < m - 1) lt -= ldcg<T>(P.uLx + i) * (wtd ? to_acc(P.a0x[i]) : Acc(1));
    if (r > 0) lt += ldcg<T>(P.uLx + i - 1) * (wtd ? to_acc(P.a0x[i - 1]) : Acc(1));
    if (c < m - 1) lt -= ldcg<T>(P.uLy + i) * (wtd ? to_acc(P.a0y[i]) : Acc(1));
    if (c > 0) lt += ldcg<T>(P.uLy + i - m) * (wtd ? to_acc(P.a0y[i - m]) : Acc(1));
    Acc vt = At[j] + sg * inv_beta * lt;
    if (!init) vt -= ba * ldcg<T>(P.v + i);
    P.v[i] = store_cast<T, Acc>(vt);
    s_v += vt * vt;
  }
  red[0] = (double)s_v;
  red[1] = 0.0;
  red[2] = 0.0;
}

// Scalar work of the block that finished a problem's last tile.
__device__ __forceinline__ void lsqr_finish_F(const LsqrCtl& ctl, LsqrState* st, bool init, int it,
                                              const double (&tot)[3]) {
  LsqrState S = load_state(st);
  const double beta_new = sqrt(tot[0]);
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
      S.dnorm2 += tot[2] / (S.rho_last * S.rho_last);
      const double xnorm = sqrt(tot[1]);
      const double anorm = sqrt(S.anorm2);
      const double acond = anorm * sqrt(S.dnorm2);
      const double rnorm = S.t_rnorm, arnorm = S.t_arnorm;
      int stop = 0;
      if (rnorm <= ctl.btol * S.bnorm + ctl.atol * anorm * xnorm) stop = 1;
      else if (anorm > 0.0 && rnorm > 0.0 && arnorm <= ctl.atol * anorm * rnorm) stop = 2;
      else if (acond >= ctl.conlim) stop = 3;
      else if (k >= ctl.maxit) stop = 4;
      if (stop) { S.done = 1; S.stop = stop; S.its = k; }
    }
    S.beta = beta_new;
    S.it = it;
  }
  *st = S;
}

__device__ __forceinline__ void lsqr_finish_B(LsqrState* st, bool init, const double (&tot)[3]) {
  LsqrState S = load_state(st);
  const double alpha_new = sqrt(tot[0]);
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
    const double rho = sqrt(S.rhobar * S.rhobar + beta * beta);
    const double c = S.rhobar / rho, s = beta / rho;
    const double theta = s * alpha_new;
    S.rhobar = -c * alpha_new;
    const double phi = c * S.phibar;
    S.phibar = s * S.phibar;
    S.phi_rho = phi / rho;
    S.theta_rho = theta / rho;
    S.rho_last = rho;
    S.t_rnorm = S.phibar;
    S.t_arnorm = S.phibar * alpha_new * fabs(c);
    S.alpha = alpha_new;
  }
  *st = S;
}

__device__ __forceinline__ bool all_done(const LsqrCtl& ctl) {
  for (int p = 0; p < ctl.nprob; ++p)
    if (__ldcg(&ctl.st[p].done) == 0) return false;
  return true;
}

template <typename T, typename Acc>
__global__ void __launch_bounds__(256) k_lsqr(const LsqrProb<T, Acc>* __restrict__ probs, LsqrCtl ctl) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Acc* sm = reinterpret_cast<Acc*>(smem_raw);
  __shared__ double scratch[3 * 32];
  __shared__ int s_flag;
  __shared__ LsqrState s_st;
  const unsigned G = gridDim.x;
  // phase 0: F(init), B(init); then F_i, B_i for i = 1, 2, ... until every
  // problem has stopped (decided at each barrier by the last block to arrive)
  auto decide = [&]() -> int { return all_done(ctl) ? 1 : 0; };
  for (int it = 0;; ++it) {
    for (int half = 0; half < 2; ++half) {
      const bool isF = (half == 0);
      for (int tile = blockIdx.x; tile < ctl.ntiles; tile += G) {
        const int p = ctl.tile_prob[tile];
        const LsqrProb<T, Acc>& P = probs[p];
        __syncthreads();
        if (threadIdx.x == 0 && threadIdx.y == 0) s_st = load_state(&ctl.st[p]);
        __syncthreads();
        if (s_st.done) continue;
        const int tl = tile - P.tile_begin;
        const int r0 = (tl % P.nt) * TM, c0 = (tl / P.nt) * TN;
        double red[3];
        if (isF) lsqr_pass_F<T, Acc>(P, s_st, it == 0, it == 1, r0, c0, sm, red);
        else lsqr_pass_B<T, Acc>(P, s_st, it == 0, r0, c0, sm, red);
        if (finish_tile<3>(red, ctl.part, ctl.cnt, tile, p, P.ntiles, scratch, &s_flag)) {
          if (threadIdx.y == 0) {
            double tot[3];
            problem_sum<3>(ctl.part, P.tile_begin, P.ntiles, tot);
            if (threadIdx.x == 0) {
              if (isF) lsqr_finish_F(ctl, &ctl.st[p], it == 0, it, tot);
              else lsqr_finish_B(&ctl.st[p], it == 0, tot);
              ctl.cnt[p] = 0;
              __threadfence();
            }
          }
        }
      }
      int stop = 0;
      if (!grid_sync(ctl.gb, G, ctl.limit_ns, decide, &stop)) return;
      if (stop) return;
    }
  }
}

}  // namespace db
