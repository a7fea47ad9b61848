// GCV choice of the regularisation parameter (Sec. 3, Eq. (xgamma), Eq. (GCV)).
//
// GCV(gamma) = ||A x_gamma - b||^2 / (n - tr(A A_gamma^{-1} A^T))^2.
// Projected form (this library's choice; the paper's dense GSVD does not
// scale past m ~ 64):
//  * numerator: x_gamma restricted to span(V), V = orthonormal basis of
//    K_k(A^T A, A^T b) (Lanczos on A^T A with two classical Gram-Schmidt
//    passes per step) plus orth(D^T c) when the shift c is non-zero.
//    G_A = V^T A^T A V, G_D = V^T D^T D V, g_A = V^T A^T b, g_D = V^T D^T c
//    are accumulated as the basis grows (double) and the small problem is
//    solved for each trial gamma in double (see k_gcv_select).
//  * exact mode (levels with at most `exact_max_pixels` pixels): V = I, i.e.
//    the dense matrices of the pair, and the exact trace -- the paper's
//    definition.
//  * trace (projected mode): the same pair under periodic boundary conditions,
//      T(gamma) = sum_w 1 / (1 + gamma s rho_w),  rho_w = l(w) / |K(w)|^2,
//    K = DFT of the level's interior stencil, l = 4 sin^2(pi j1/m) + 4 sin^2(pi j2/m),
//    s = mean squared IRLS weight (1 for an unweighted pair).
//  * selection: 50-point log grid on [1e-10, 1e2] (the side holding the
//    minimum widened by 4 decades, at most twice), then Brent's minimiser
//    (golden section + parabolic steps, Brent 1973) on log10(gamma).
#pragma once
#include "outer.cuh"
#include <cooperative_groups.h>

namespace db {

// ---- symbol of the level's interior stencil ---------------------------------
// Kf[t][j] = sum_k B_t[m/2][k] exp(+2 pi i j (dlo + k) / m)  (complex double)
__global__ void k_band_dft(int m, int dlo, int w, int nterms, const double* __restrict__ B,
                           double2* __restrict__ Kf) {
  size_t total = (size_t)nterms * m;
  const int rmid = m / 2;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    int j = (int)(i % m), t = (int)(i / m);
    double re = 0, im = 0;
    for (int k = 0; k < w; ++k) {
      double bv = B[((size_t)t * m + rmid) * w + k];
      if (bv == 0.0) continue;
      long long d = (long long)dlo + k;
      long long ph = ((long long)j * d) % m;        // exact phase index
      if (ph < 0) ph += m;
      double s, c;
      sincospi(2.0 * (double)ph / (double)m, &s, &c);
      re += bv * c;
      im += bv * s;
    }
    Kf[i] = make_double2(re, im);
  }
}

// rho[j1 + j2 m] = l(j1, j2) / |sum_t Kr_t(j1) Kc_t(j2)|^2 (float; +inf where K = 0)
__global__ void k_symbol_rho(int m, int nterms, const double2* __restrict__ Kr, const double2* __restrict__ Kc,
                             float* __restrict__ rho) {
  size_t n = (size_t)m * m;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    int j1 = (int)(i % m), j2 = (int)(i / m);
    double re = 0, im = 0;
    for (int t = 0; t < nterms; ++t) {
      double2 a = Kr[(size_t)t * m + j1], b = Kc[(size_t)t * m + j2];
      re += a.x * b.x - a.y * b.y;
      im += a.x * b.y + a.y * b.x;
    }
    double k2 = re * re + im * im;
    double s1 = sinpi((double)j1 / m), s2 = sinpi((double)j2 / m);
    double l = 4.0 * s1 * s1 + 4.0 * s2 * s2;
    rho[i] = k2 > 0.0 ? (float)(l / k2) : __int_as_float(0x7f800000);
  }
}

// ---- Krylov basis helpers ------------------------------------------------------
// part[v * nchunks + chunk] = sum over the chunk of V_v . y   (v < nvec)
template <typename Acc>
__global__ void __launch_bounds__(256) k_mdot(size_t n, int nvec, const Acc* __restrict__ V, size_t ldv,
                                              const Acc* __restrict__ y, double* __restrict__ part) {
  __shared__ double scratch[32];
  const int v = blockIdx.y;
  const size_t chunk = (n + gridDim.x - 1) / gridDim.x;
  const size_t beg = blockIdx.x * chunk;
  const size_t end = beg + chunk < n ? beg + chunk : n;
  double acc = 0.0;
  const Acc* vv = V + (size_t)v * ldv;
  for (size_t i = beg + threadIdx.x; i < end; i += blockDim.x) acc += (double)vv[i] * (double)y[i];
  double red[1] = {acc};
  block_sum<1>(red, scratch);
  if (threadIdx.x == 0) part[(size_t)v * gridDim.x + blockIdx.x] = red[0];
}

// out[v * ostride] = sum_chunk part[v * nchunks + chunk]   (fixed order)
__global__ void k_mdot_reduce(int nvec, int nchunks, const double* __restrict__ part, double* out, int ostride) {
  const int v = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  const int lane = threadIdx.x & 31;
  if (v >= nvec) return;
  double s = 0.0;
  for (int c = lane; c < nchunks; c += 32) s += part[(size_t)v * nchunks + c];
  s = warp_sum(s);
  if (lane == 0) out[(size_t)v * ostride] = s;
}

// y -= sum_{v < nvec} h[v * hstride] V_v
template <typename Acc>
__global__ void k_maxpy(size_t n, int nvec, const Acc* __restrict__ V, size_t ldv, const double* __restrict__ h,
                        int hstride, Acc* __restrict__ y) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    Acc s = y[i];
    for (int v = 0; v < nvec; ++v) s -= (Acc)h[(size_t)v * hstride] * V[(size_t)v * ldv + i];
    y[i] = s;
  }
}

// y = x * (1 / sqrt(*nrm2))
template <typename Acc>
__global__ void k_scale_inv_sqrt(size_t n, const Acc* __restrict__ x, const double* nrm2, Acc* __restrict__ y) {
  const double inv = 1.0 / sqrt(*nrm2);
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    y[i] = (Acc)((double)x[i] * inv);
}

// Convert a storage-typed vector to Acc, optionally c = a - b (planes).
template <typename T, typename Acc>
__global__ void k_to_acc(size_t n, const T* __restrict__ a, const T* __restrict__ b, Acc* __restrict__ y) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    y[i] = (Acc)(to_acc(a[i]) - (b ? to_acc(b[i]) : (decltype(to_acc(a[i])))0));
}

// x = L^T (w o q) on Acc planes (weights may be null): used for D^T c.
template <typename Acc, typename T>
__global__ void k_Lt_w(int m, const Acc* __restrict__ qx, const Acc* __restrict__ qy, const T* __restrict__ wx,
                       const T* __restrict__ wy, Acc* __restrict__ x) {
  size_t n = (size_t)m * m;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    int r = (int)(i % m), c = (int)(i / m);
    auto W = [&](const T* p, size_t k) -> Acc { return p ? (Acc)to_acc(p[k]) : Acc(1); };
    Acc s = 0;
    if (r < m - 1) s -= W(wx, i) * qx[i];
    if (r > 0) s += W(wx, i - 1) * qx[i - 1];
    if (c < m - 1) s -= W(wy, i) * qy[i];
    if (c > 0) s += W(wy, i - m) * qy[i - m];
    x[i] = s;
  }
}

// ---- fused Krylov-basis kernels ------------------------------------------------
// Each block owns one contiguous chunk of the vectors; per-chunk partial sums
// are kept as double-float pairs (float hi + float lo, error-free TwoSum, see
// df_add) in part[slot * nchunks + chunk], and k_part_reduce adds the chunks
// of every output slot in a fixed order, one warp per slot.
constexpr int VCH_E = 8;                 // elements per thread per chunk
constexpr int VCH_THREADS = 256;
constexpr int VCH_CHUNK = VCH_E * VCH_THREADS;
enum VchunkMode { VCH_UPDATE = 1, VCH_DOTS = 2, VCH_NORM = 4 };

// x -= sum_{i<nrows} coef[i*cstride] V_i (VCH_UPDATE); then the chunk
// partials of V_i . x for i < nrows into slots 0..nrows-1 (VCH_DOTS) and/or
// of x . x into slot nrows (VCH_NORM), summed by k_part_reduce with
// RedRows. Float vectors only (the Krylov basis is held in working
// precision); part needs (nrows + 1) * gridDim.x float2.
__global__ void __launch_bounds__(VCH_THREADS) k_vchunk(size_t n, int nrows, const float* __restrict__ V, size_t ldv,
    const double* __restrict__ coef, int cstride, float* __restrict__ x, int mode, float2* __restrict__ part,
    int E) {
  __shared__ float xs[VCH_CHUNK];
  __shared__ float cs[512];
  const int nch = gridDim.x, ch = blockIdx.x;
  const int CH = E * VCH_THREADS;
  const size_t beg = (size_t)ch * CH;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = VCH_THREADS / 32;
  if (mode & VCH_UPDATE)
    for (int i = tid; i < nrows; i += VCH_THREADS) cs[i] = (float)coef[(size_t)i * cstride];
  __syncthreads();
  float nhi = 0.f, nlo = 0.f;
  for (int k = 0; k < E; ++k) {
    const int le = k * VCH_THREADS + tid;
    const size_t e = beg + le;
    float xv = 0.f;
    if (e < n) {
      xv = x[e];
      if (mode & VCH_UPDATE) {
        for (int i = 0; i < nrows; ++i) xv -= cs[i] * V[(size_t)i * ldv + e];
        x[e] = xv;
      }
      df_fma(nhi, nlo, xv, xv);
    }
    xs[le] = xv;
  }
  __syncthreads();
  if (mode & VCH_DOTS) {
    for (int i = wid; i < nrows; i += nw) {
      const float* vi = V + (size_t)i * ldv + beg;
      float hi = 0.f, lo = 0.f;
      for (int le = lane; le < CH; le += 32) {
        if (beg + le >= n) break;
        df_fma(hi, lo, vi[le], xs[le]);
      }
      const float2 r = warp_df_pair(hi, lo);
      if (lane == 0) part[(size_t)i * nch + ch] = r;
    }
  }
  if (mode & VCH_NORM) {
    const float2 r = warp_df_pair(nhi, nlo);
    __shared__ float2 wn[8];
    if (lane == 0) wn[wid] = r;
    __syncthreads();
    if (tid == 0) {
      float hi = 0.f, lo = 0.f;
      for (int w = 0; w < nw; ++w) df_add(hi, lo, wn[w].x, wn[w].y);
      part[(size_t)nrows * nch + ch] = make_float2(hi, lo);
    }
  }
}

// One Gram column for the basis vector vj against rows V_0..V_{nr-1} and
// itself, stored as column jout (jout >= nr): with y = L^T diag(w^2) L vj
// (computed here),
//   GA[i*ld + jout] = V_i . t, GD[i*ld + jout] = V_i . y   (i < nr),
//   GA[jout*ld + jout] = vj . t, GD[jout*ld + jout] = vj . y,
//   gA[jout] = atb . vj, gD[jout] = dtc . vj (dtc may be null -> 0),
// as chunk partials in slots 2i (A part) and 2i+1 (D part) for the rows
// i = 0..nr (row nr is vj) and i = nr+1 (the g entries), summed by
// k_part_reduce with RedGramCol. t == null computes only the D part (GD, gD),
// for a basis whose GA is known.
template <typename T>
__global__ void __launch_bounds__(VCH_THREADS) k_gram_col(int m, int nr, const float* __restrict__ vj, int jout,
    const float* __restrict__ V, const float* __restrict__ t, const T* __restrict__ wx, const T* __restrict__ wy,
    const float* __restrict__ atb, const float* __restrict__ dtc, float2* __restrict__ part, int E) {
  __shared__ float ts[VCH_CHUNK];
  __shared__ float ys[VCH_CHUNK];
  const size_t n = (size_t)m * m;
  const int nch = gridDim.x, ch = blockIdx.x;
  const int CH = E * VCH_THREADS;
  const size_t beg = (size_t)ch * CH;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = VCH_THREADS / 32;
  const bool with_a = (t != nullptr);
  for (int k = 0; k < E; ++k) {
    const int le = k * VCH_THREADS + tid;
    const size_t i = beg + le;
    float tv = 0.f, yv = 0.f;
    if (i < n) {
      if (with_a) tv = t[i];
      const int r = (int)(i % m), c = (int)(i / m);
      const float xv = vj[i];
      auto W = [&](const T* p, size_t q) -> float { return p ? (float)to_acc(p[q]) : 1.f; };
      if (r < m - 1) { const float w = W(wx, i); yv -= w * w * (vj[i + 1] - xv); }
      if (r > 0) { const float w = W(wx, i - 1); yv += w * w * (xv - vj[i - 1]); }
      if (c < m - 1) { const float w = W(wy, i); yv -= w * w * (vj[i + m] - xv); }
      if (c > 0) { const float w = W(wy, i - m); yv += w * w * (xv - vj[i - m]); }
    }
    ts[le] = tv;
    ys[le] = yv;
  }
  __syncthreads();
  const int nrows = nr + 1;            // rows V_0..V_{nr-1} and vj itself
  // rows 0..nr: two dots each (slots 2i, 2i+1); row nr+1: atb.vj and dtc.vj
  for (int i = wid; i <= nrows; i += nw) {
    float h1 = 0.f, l1 = 0.f, h2 = 0.f, l2 = 0.f;
    const float* vi = i < nr ? V + (size_t)i * n : vj;
    for (int le = lane; le < CH; le += 32) {
      if (beg + le >= n) break;
      float p1, q1, p2, q2;
      if (i < nrows) { const float vv = vi[beg + le]; p1 = vv; q1 = ts[le]; p2 = vv; q2 = ys[le]; }
      else { const float vv = vj[beg + le]; p1 = with_a ? atb[beg + le] : 0.f; q1 = vv; p2 = dtc ? dtc[beg + le] : 0.f; q2 = vv; }
      df_fma(h1, l1, p1, q1);
      df_fma(h2, l2, p2, q2);
    }
    const float2 r1 = warp_df_pair(h1, l1), r2 = warp_df_pair(h2, l2);
    if (lane == 0) {
      part[(size_t)(2 * i) * nch + ch] = r1;
      part[(size_t)(2 * i + 1) * nch + ch] = r2;
    }
  }
}

// ---- G_D of a whole basis at once ------------------------------------------------
// G_D = V^T L^T diag(w^2) L V = Z^T Z with Z = diag(w) L V, the 2n x kk matrix
// of the basis's weighted gradients. One pass over V: each block takes a
// contiguous pixel range, forms the rows of Z of its pixels (x- and y-plane
// components) in shared memory, SK_PC pixels at a time, and accumulates
// Z_rows^T Z_rows in registers: thread t owns the SK_TI x SK_TI output block
// (bi, bj), bi <= bj, of the upper triangle (FP32 products, FP32 sums over the
// block's pixel range). The per-block partials are added in double, in block
// order, by k_gram_dtd_reduce. The result depends only on V, the weights and
// the pixel ranges, so a cached basis and a rebuilt one give the same G_D.
constexpr int SK_TI = 11;                          // outputs per thread and dimension
constexpr int SK_NB = 15;                          // block rows (kk <= 165)
constexpr int SK_KMAX = SK_TI * SK_NB;
constexpr int SK_NPAIR = SK_NB * (SK_NB + 1) / 2;  // 120 upper-triangle blocks
constexpr int SK_THREADS = 128;
constexpr int SK_PC = 32;                          // pixels per shared-memory stage
constexpr int SK_SLOTS = SK_NPAIR * SK_TI * SK_TI;

__device__ __forceinline__ void sk_pair(int t, int nb, int& bi, int& bj) {
  bi = 0;
  while (t >= nb - bi) { t -= nb - bi; ++bi; }
  bj = bi + t;
}

// part[blk * nslot + e * npair + t] = partial of entry e = ii * SK_TI + jj of
// block pair t, nslot = npair * SK_TI^2, npair = nb (nb + 1) / 2.
template <typename T>
__global__ void __launch_bounds__(SK_THREADS) k_gram_dtd(int m, int kk, const float* __restrict__ V,
    const T* __restrict__ wx, const T* __restrict__ wy, int ppb, float* __restrict__ part) {
  __shared__ float zs[2 * SK_PC][SK_KMAX];
  const size_t n = (size_t)m * m;
  const int nb = (kk + SK_TI - 1) / SK_TI;
  const int npair = nb * (nb + 1) / 2;
  const int kpad = nb * SK_TI;
  const int t = threadIdx.x;
  const bool active = t < npair;
  int bi = 0, bj = 0;
  if (active) sk_pair(t, nb, bi, bj);
  float acc[SK_TI][SK_TI];
#pragma unroll
  for (int a = 0; a < SK_TI; ++a)
#pragma unroll
    for (int b = 0; b < SK_TI; ++b) acc[a][b] = 0.f;
  const size_t p0 = (size_t)blockIdx.x * ppb;
  const size_t p1 = (p0 + (size_t)ppb < n) ? p0 + (size_t)ppb : n;
  for (size_t pc = p0; pc < p1; pc += SK_PC) {
    __syncthreads();                 // the previous stage's rows are consumed
    for (int idx = t; idx < SK_PC * kpad; idx += SK_THREADS) {
      const int r = idx & (SK_PC - 1), j = idx / SK_PC;
      const size_t i = pc + r;
      float zx = 0.f, zy = 0.f;
      if (j < kk && i < p1) {
        const float* vj = V + (size_t)j * n;
        const int row = (int)(i % m), col = (int)(i / m);
        const float xv = vj[i];
        if (row < m - 1) zx = (wx ? (float)to_acc(wx[i]) : 1.f) * (vj[i + 1] - xv);
        if (col < m - 1) zy = (wy ? (float)to_acc(wy[i]) : 1.f) * (vj[i + m] - xv);
      }
      zs[r][j] = zx;
      zs[SK_PC + r][j] = zy;
    }
    __syncthreads();
    if (active) {
#pragma unroll 2
      for (int r = 0; r < 2 * SK_PC; ++r) {
        float a[SK_TI], b[SK_TI];
#pragma unroll
        for (int q = 0; q < SK_TI; ++q) {
          a[q] = zs[r][bi * SK_TI + q];
          b[q] = zs[r][bj * SK_TI + q];
        }
#pragma unroll
        for (int x = 0; x < SK_TI; ++x)
#pragma unroll
          for (int y = 0; y < SK_TI; ++y) acc[x][y] = fmaf(a[x], b[y], acc[x][y]);
      }
    }
  }
  if (active) {
    const size_t nslot = (size_t)npair * SK_TI * SK_TI;
    float* out = part + (size_t)blockIdx.x * nslot + t;
#pragma unroll
    for (int x = 0; x < SK_TI; ++x)
#pragma unroll
      for (int y = 0; y < SK_TI; ++y) out[(size_t)(x * SK_TI + y) * npair] = acc[x][y];
  }
}

// GD[i * ld + j] (i <= j < kk) = sum over the nblk block partials, in block
// order: 32 slots per block of 256 threads, eight groups of blocks summed in
// parallel and combined in group order.
__global__ void __launch_bounds__(256) k_gram_dtd_reduce(int nblk, int kk, const float* __restrict__ part,
                                                         double* __restrict__ GD, int ld) {
  __shared__ double red[8][32];
  const int nb = (kk + SK_TI - 1) / SK_TI;
  const int npair = nb * (nb + 1) / 2;
  const int nslot = npair * SK_TI * SK_TI;
  const int lane = threadIdx.x & 31, g = threadIdx.x >> 5;
  const int s = blockIdx.x * 32 + lane;
  double acc = 0.0;
  if (s < nslot)
    for (int c = g; c < nblk; c += 8) acc += (double)__ldg(part + (size_t)c * nslot + s);
  red[g][lane] = acc;
  __syncthreads();
  if (g == 0 && s < nslot) {
    double tot = 0.0;
#pragma unroll
    for (int k = 0; k < 8; ++k) tot += red[k][lane];
    const int e = s / npair, tp = s - e * npair;
    int bi, bj;
    sk_pair(tp, nb, bi, bj);
    const int i = bi * SK_TI + e / SK_TI, j = bj * SK_TI + e % SK_TI;
    if (i <= j && j < kk) GD[(size_t)i * ld + j] = tot;
  }
}

// ---- chunk-partial reduction -----------------------------------------------
// Output slot s of a chunk kernel is the sum of part[s * nch + c] over the
// chunks c; one warp per slot, lane l adding chunks l, l + 32, ... (batches of
// RED_BATCH loads) and the warp butterfly combining the lanes, so the result
// depends only on the partials and nch. Map::dst(s) gives the destination of
// slot s (null: not stored).
constexpr int RED_BATCH = 8;
template <class Map>
__global__ void __launch_bounds__(256) k_part_reduce(int nslot, int nch, const float2* __restrict__ part, Map map) {
  const int lane = threadIdx.x & 31;
  const int s = blockIdx.x * 8 + (threadIdx.x >> 5);
  if (s >= nslot) return;
  double* d = map.dst(s);
  if (d == nullptr) return;
  const float2* p = part + (size_t)s * nch;
  float hi = 0.f, lo = 0.f;
  for (int c0 = 0; c0 < nch; c0 += 32 * RED_BATCH) {
    float2 q[RED_BATCH];
#pragma unroll
    for (int k = 0; k < RED_BATCH; ++k) {
      const int c = c0 + k * 32 + lane;
      q[k] = c < nch ? p[c] : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int k = 0; k < RED_BATCH; ++k) df_add(hi, lo, q[k].x, q[k].y);
  }
  const float2 r = warp_df_pair(hi, lo);
  if (lane == 0) *d = (double)r.x + (double)r.y;
}

// k_vchunk slots r0 .. : row r < nrows -> out[r * ostride], r == nrows -> *outnorm
struct RedRows {
  int r0, nrows, ostride;
  double* out;
  double* outnorm;
  __device__ double* dst(int s) const {
    const int r = r0 + s;
    return r < nrows ? out + (size_t)r * ostride : outnorm;
  }
};

// k_gram_col slots (see there)
struct RedGramCol {
  int nr, jout, ld, with_a;
  double *GA, *GD, *gA, *gD;
  __device__ double* dst(int s) const {
    const int i = s >> 1;
    const bool a_part = (s & 1) == 0;
    if (a_part && !with_a) return nullptr;
    if (i <= nr) {
      const int row = i < nr ? i : jout;
      return (a_part ? GA : GD) + (size_t)row * ld + jout;
    }
    return (a_part ? gA : gD) + jout;
  }
};

// ---- exact mode: dense matrices of the pair (n <= a few hundred) ------------
// A[(r + c m), (r' + c' m)] = sum_t Cr_t[r, r'] Cc_t[c, c'], C[r, s] = B[r][(s - r - dlo) mod m].
__device__ __forceinline__ double band_entry(const double* B, int t, int m, int dlo, int w, int r, int s) {
  const int k = wrap(s - r - dlo, m);
  return k < w ? B[((size_t)t * m + r) * w + k] : 0.0;
}

__global__ void k_dense_blur(int m, int nterms, int dlo, int w, const double* __restrict__ Br,
                             const double* __restrict__ Bc, double* __restrict__ Ad) {
  const int n = m * m;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < (size_t)n * n;
       idx += (size_t)gridDim.x * blockDim.x) {
    const int row = (int)(idx / n), col = (int)(idx % n);
    const int r = row % m, c = row / m, r2 = col % m, c2 = col / m;
    double v = 0.0;
    for (int t = 0; t < nterms; ++t)
      v += band_entry(Br, t, m, dlo, w, r, r2) * band_entry(Bc, t, m, dlo, w, c, c2);
    Ad[idx] = v;
  }
}

// G[i][j] = sum_l A[l][i] A[l][j]  (full n x n, row-major, leading dimension ld)
__global__ void k_gram_dense(int n, const double* __restrict__ Ad, double* __restrict__ G, int ld) {
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < (size_t)n * n;
       idx += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(idx / n), j = (int)(idx % n);
    double s0 = 0.0, s1 = 0.0;
    int l = 0;
    for (; l + 1 < n; l += 2) { s0 += Ad[(size_t)l * n + i] * Ad[(size_t)l * n + j]; s1 += Ad[(size_t)(l + 1) * n + i] * Ad[(size_t)(l + 1) * n + j]; }
    if (l < n) s0 += Ad[(size_t)l * n + i] * Ad[(size_t)l * n + j];
    G[(size_t)i * ld + j] = s0 + s1;
  }
}

// (L^T diag(w^2) L)[i][j] from the 5-point stencil (weights may be null).
template <typename T>
__global__ void k_dense_DtD(int m, const T* __restrict__ wx, const T* __restrict__ wy, double* __restrict__ G, int ld) {
  const int n = m * m;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < (size_t)n * n;
       idx += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(idx / n), j = (int)(idx % n);
    const int r = i % m, c = i / m;
    auto X = [&](int k) { return k == j ? 1.0 : 0.0; };
    auto W = [&](const T* p, int k) { return p ? (double)to_acc(p[k]) : 1.0; };
    double s = 0.0;
    const double xv = X(i);
    if (r < m - 1) { const double ww = W(wx, i); s -= ww * ww * (X(i + 1) - xv); }
    if (r > 0) { const double ww = W(wx, i - 1); s += ww * ww * (xv - X(i - 1)); }
    if (c < m - 1) { const double ww = W(wy, i); s -= ww * ww * (X(i + m) - xv); }
    if (c > 0) { const double ww = W(wy, i - m); s += ww * ww * (xv - X(i - m)); }
    G[(size_t)i * ld + j] = s;
  }
}

// g = Ad^T b (Ad row-major n x n), double
__global__ void k_dense_matvecT(int n, const double* __restrict__ Ad, const double* __restrict__ b, double* g) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int l = 0; l < n; ++l) s += Ad[(size_t)l * n + j] * b[l];
    g[j] = s;
  }
}

// y = a - b (b may be null) in double, from storage-precision inputs.
template <typename T>
__global__ void k_diff_to_double(size_t n, const T* __restrict__ a, const T* __restrict__ b, double* __restrict__ y) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    y[i] = (double)to_acc(a[i]) - (b ? (double)to_acc(b[i]) : 0.0);
}

template <typename Acc>
__global__ void k_to_double(size_t n, const Acc* __restrict__ x, double* __restrict__ y) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    y[i] = (double)x[i];
}

// ---- the small problem and the selection (one block) --------------------------
// With M = G_A + G_D = R R^T (Cholesky), C = R^{-1} G_A R^{-T} = Q T Q^T
// (Householder, T tridiagonal) and p_A = Q^T R^{-1} g_A, p_D = Q^T R^{-1} g_D,
// the trial solution of (G_A + gamma G_D) y = g_A + gamma g_D is
// y = R^{-T} Q w with ((1 - gamma) T + gamma I) w = p_A + gamma p_D (a
// tridiagonal SPD system per gamma, one Thomas sweep); the residual is
// evaluated without cancellation as gamma^2 u^T T u + r0^2. The trace is either the symbol
// trace (projected mode) or, when the basis is the whole space (exact mode,
// tiny levels), sum_j lam_j / (lam_j + gamma (1 - lam_j)) over the
// eigenvalues of T (bisection with Sturm counts).
//
// Layout: the k x k working matrix (M, then R, then C and the reduction to
// T) lives in shared memory when k <= SEL_SMEM_K (row pitch k|1, so a warp
// reading a column, or the same column index of consecutive rows, touches
// distinct banks); the two k x k intermediates of the congruence go to the
// global work buffer. FP64 costs ~64 cycles of pipe time per warp
// instruction on this part, so reductions run only in the warps that hold
// data and the tridiagonalisation updates the lower triangle only.
struct GcvSelectArgs {
  int kk;                 // basis dimension
  int ld;                 // leading dimension of GA, GD
  const double* GA;       // upper triangle valid (i <= j)
  const double* GD;
  const double* gA;
  const double* gD;
  double bnorm2;
  double n;               // pixel count of the level
  double s;               // weight scale of the trace
  const float* rho;       // [npix] symbol ratios (projected mode)
  int npix;
  int exact;              // 1: trace from the eigenvalues of T
  double lo, hi, tolx;
  int npts, max_ext;
  const double* trace_tab;  // projected mode: traces on the first grid (npts values), or null
  int kshift;             // >= 0: basis vector kk-1 is stored at row/column kshift of GA, GD, gA, gD
  double* work;           // >= sel_work_doubles(kk)
  double* out;            // out[0] = gamma, out[1] = extensions, out[2] = GCV value
};

constexpr int SEL_THREADS = 512;
constexpr int SEL_MAXPTS = 64;
constexpr int SEL_SMEM_K = 162;   // largest basis whose matrix is kept in shared memory
constexpr int SEL_NVEC = 10;      // k-vectors in shared memory

__host__ __device__ inline int sel_lds(int kk) { return kk | 1; }
// Global work of one selection: (matrix if not in shared memory), X, C, and
// the per-grid-point scratch (2 kk per point for the single-block selector,
// 4 kk for the cluster selector, whose X takes kk^2 + 2 kk).
inline size_t sel_work_doubles(int kk) {
  return (kk <= SEL_SMEM_K ? 0 : (size_t)kk * sel_lds(kk)) + (size_t)2 * kk * kk + (size_t)4 * SEL_MAXPTS * kk;
}
// Dynamic shared memory of k_gcv_select: the k-vectors, then (k <= SEL_SMEM_K)
// the working matrix.
inline size_t sel_smem_bytes(int kk) {
  size_t v = (size_t)SEL_NVEC * kk * sizeof(double);
  if (kk <= SEL_SMEM_K) v += (size_t)kk * sel_lds(kk) * sizeof(double);
  return v;
}

// 1/x in double from a float reciprocal refined by two Newton steps
// (22 -> 44 -> 88 bits, i.e. correctly rounded to within an ulp); an FP64
// divide costs several hundred cycles of latency on this part.
__device__ __forceinline__ double rcp_d(double x) {
  const double ax = fabs(x);
  if (!(ax > 1e-30 && ax < 1e30)) return 1.0 / (ax > 1e-300 ? x : 1e-300);
  double y = (double)__frcp_rn((float)x);
  y = y * (2.0 - x * y);
  y = y * (2.0 - x * y);
  return y;
}

// 1/sqrt(x) in double: float estimate, then two Newton steps
// y <- y (3 - x y^2) / 2 (each roughly doubles the correct bits).
__device__ __forceinline__ double rsqrt_d(double x) {
  if (!(x > 1e-30 && x < 1e30)) return 1.0 / sqrt(x > 1e-300 ? x : 1e-300);
  double y = (double)rsqrtf((float)x);
  y = y * (1.5 - 0.5 * x * y * y);
  y = y * (1.5 - 0.5 * x * y * y);
  return y;
}

// Block sum of N doubles over nact elements that the threads hold strided
// (element i in thread i mod blockDim.x): only threads [0, min(nact,
// blockDim.x)) hold values; the other threads pass zeros and skip the FP64
// shuffles. Result in every thread. sh >= 32 N.
template <int N>
__device__ __forceinline__ void sel_sumN(double (&v)[N], int nact, double* sh) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int nw = min((nact + 31) >> 5, (int)(blockDim.x >> 5));
  if (wid < nw) {
#pragma unroll
    for (int k = 0; k < N; ++k) v[k] = warp_sum(v[k]);
  }
  __syncthreads();
  if (lane == 0 && wid < nw) {
#pragma unroll
    for (int k = 0; k < N; ++k) sh[k * 32 + wid] = v[k];
  }
  __syncthreads();
  if (wid == 0) {
#pragma unroll
    for (int k = 0; k < N; ++k) {
      double t = lane < nw ? sh[k * 32 + lane] : 0.0;
      t = warp_sum(t);
      if (lane == 0) sh[k * 32] = t;
    }
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < N; ++k) v[k] = sh[k * 32];
  __syncthreads();
}

__device__ double sel_block_sum(double v, double* sh) {
  double t[1] = {v};
  sel_sumN<1>(t, blockDim.x, sh);
  return t[0];
}

// Solve ((1 - gamma) T + gamma I) u = f by one Thomas sweep (T symmetric
// tridiagonal: diagonal d, off-diagonal e; the matrix is SPD for gamma > 0
// and for gamma = 0 when T is). cw is scratch of length kk. One thread.
__device__ void sel_tri_solve(int kk, const double* d, const double* e, const double* f, double gamma,
                              double* cw, double* u, double shift = 0.0) {
  const double a = 1.0 - gamma;
  const double diag_add = gamma + shift;
  double piv = a * d[0] + diag_add;
  double inv = rcp_d(piv);
  cw[0] = (kk > 1) ? (a * e[0]) * inv : 0.0;
  u[0] = f[0] * inv;
  for (int i = 1; i < kk; ++i) {
    const double off = a * e[i - 1];
    piv = a * d[i] + diag_add - off * cw[i - 1];
    inv = rcp_d(piv);
    cw[i] = (i + 1 < kk) ? (a * e[i]) * inv : 0.0;
    u[i] = (f[i] - off * u[i - 1]) * inv;
  }
  for (int i = kk - 2; i >= 0; --i) u[i] -= cw[i] * u[i + 1];
}

// Numerator ||A V y_gamma - b||^2 = gamma^2 u^T T u + r0^2 with
// ((1 - gamma) T + gamma I) u = f, f = p_A + p_D - T^{-1} p_A: the
// gamma-dependent part is a quadratic form in T (no cancellation against
// ||b||^2). One thread.
__device__ double sel_numerator(int kk, const double* d, const double* e, const double* f, double r02,
                                double gamma, double* cw, double* u) {
  sel_tri_solve(kk, d, e, f, gamma, cw, u);
  double q = 0.0;
  for (int i = 0; i < kk; ++i) {
    double tu = d[i] * u[i];
    if (i > 0) tu += e[i - 1] * u[i - 1];
    if (i + 1 < kk) tu += e[i] * u[i + 1];
    q += u[i] * tu;
  }
  return gamma * gamma * q + r02;
}

// 2^(-e) with e the binary exponent of x (x finite, nonzero): multiplying by
// it is exact and brings |x| into [0.5, 1).
__device__ __forceinline__ double exp2_neg_exponent(double x) {
  const long long bits = __double_as_longlong(x);
  const int e = (int)((bits >> 52) & 0x7ff) - 1022;
  return __longlong_as_double((long long)(1023 - e) << 52);
}

// Numerator gamma^2 u^T T u + r0^2 with ((1-gamma) T + gamma I) u = f, by
// the LDL^T elimination written through the leading minors
//   D_i = b_i D_{i-1} - a_i^2 D_{i-2},  pivot_i = D_i / D_{i-1},
// so the sequential recurrences carry one or two FP64 operations per row and
// every reciprocal is taken in parallel afterwards (a single thread issuing
// FP64 costs ~64 cycles per instruction here, whatever the dependencies).
// (D_i, D_{i-1}) are rescaled together by a power of two every 4 rows, which
// leaves the pivots unchanged. The elimination and its subtractions are those
// of a Thomas sweep. Warp 0 runs the recurrences while warps 1.. sum the
// symbol trace (projected mode); all threads call it. wk: 3 kk doubles.
// The single-block selector (exact mode on the tiny levels, and the fallback
// when no cluster fits) uses this one-directional form; the cluster selector
// uses the twisted form below.
__device__ double sel_eval_seq(const GcvSelectArgs& a, int kk, const double* dg, const double* eo, const double* f,
                               double r02, const double* lam, double gamma, double* u, double* wk, double* sh,
                               double* tr_out) {
  double* Dv = wk;            // D_i, then alpha_i = f_i / pivot_i
  double* Dp = wk + kk;       // D_{i-1} (same scaling), then beta_i = a_i / pivot_i
  double* cw = wk + 2 * kk;   // a_{i+1} / pivot_i
  const double g1 = 1.0 - gamma, g0 = gamma;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  __shared__ double s_trp[32];
  // (1) leading minors (thread 0) || trace partial sums (warps 1..)
  if (tid == 0) {
    double dm1 = 1.0, dm2 = 0.0;
    for (int i = 0; i < kk; ++i) {
      const double ai = i > 0 ? g1 * eo[i - 1] : 0.0;
      const double di = (g1 * dg[i] + g0) * dm1 - (ai * ai) * dm2;
      Dv[i] = di;
      Dp[i] = dm1;
      dm2 = dm1;
      dm1 = di;
      if ((i & 3) == 3 && di != 0.0) {
        const double sc = exp2_neg_exponent(di);
        dm1 *= sc;
        dm2 *= sc;
      }
    }
  }
  double trp = 0.0;
  if (wid > 0) {
    if (a.exact) {
      for (int j = tid - 32; j < kk; j += blockDim.x - 32) trp += lam[j] / (lam[j] + gamma * (1.0 - lam[j]));
    } else {
      const float gs = (float)(gamma * a.s);
      float sum = 0.f, comp = 0.f;
      constexpr int B = 8;
      const int nt = blockDim.x - 32;
      for (int base = tid - 32; base < a.npix; base += nt * B) {
        float r[B];
#pragma unroll
        for (int q = 0; q < B; ++q) {
          const int i = base + q * nt;
          r[q] = i < a.npix ? __ldg(a.rho + i) : -1.f;
        }
#pragma unroll
        for (int q = 0; q < B; ++q) {
          if (r[q] < 0.f) continue;
          const float term = __frcp_rn(1.0f + gs * r[q]);
          const float y = term - comp;
          const float t = sum + y;
          comp = (t - sum) - y;
          sum = t;
        }
      }
      trp = (double)sum - (double)comp;
    }
    trp = warp_sum(trp);
    if (lane == 0) s_trp[wid] = trp;
  }
  __syncthreads();
  // (2) reciprocals of the pivots, in parallel
  for (int i = tid; i < kk; i += blockDim.x) {
    const double d = Dv[i];
    const double inv = d != 0.0 ? Dp[i] * rcp_d(d) : 0.0;
    const double ai = i > 0 ? g1 * eo[i - 1] : 0.0;
    const double ci = i + 1 < kk ? g1 * eo[i] : 0.0;
    Dv[i] = f[i] * inv;
    Dp[i] = ai * inv;
    cw[i] = ci * inv;
  }
  __syncthreads();
  // (3) forward and back substitution (thread 0); trace total (warp 1)
  if (tid == 0) {
    double y = Dv[0];
    u[0] = y;
    for (int i = 1; i < kk; ++i) {
      y = Dv[i] - Dp[i] * y;
      u[i] = y;
    }
    double un = u[kk - 1];
    for (int i = kk - 2; i >= 0; --i) {
      un = u[i] - cw[i] * un;
      u[i] = un;
    }
  } else if (wid == 1) {
    const int nw = blockDim.x >> 5;
    double t = (lane >= 1 && lane < nw) ? s_trp[lane] : 0.0;
    t = warp_sum(t);
    if (lane == 0) *tr_out = t;
  }
  __syncthreads();
  // (4) u^T T u
  double q[1] = {0.0};
  for (int i = tid; i < kk; i += blockDim.x) {
    double tu = dg[i] * u[i];
    if (i > 0) tu += eo[i - 1] * u[i - 1];
    if (i + 1 < kk) tu += eo[i] * u[i + 1];
    q[0] += u[i] * tu;
  }
  sel_sumN<1>(q, kk, sh);
  return gamma * gamma * q[0] + r02;
}

// Numerator gamma^2 u^T T u + r0^2 with ((1 - gamma) T + gamma I) u = f
// (b_i the diagonal, a_i the entry coupling rows i-1 and i), by a twisted
// elimination at the middle row m: rows 0..m-1 are eliminated downwards
// (LDL^T pivots through the leading minors D_i = b_i D_{i-1} - a_i^2 D_{i-2},
// pivot D_i / D_{i-1}) while rows K-1..m+1 are eliminated upwards (UDU^T
// pivots through the trailing minors E_i = b_i E_{i+1} - a_{i+1}^2 E_{i+2}),
// row m is solved from both, and the back substitution runs outwards. The
// matrix is SPD for gamma > 0, so both sets of pivots are positive. The two
// halves are sequential recurrences run by two threads in different warps
// (separate FP64 pipes; a single thread issuing FP64 costs ~64 cycles per
// instruction here, whatever the dependencies); everything else (the
// coefficients, the reciprocals of the pivots, u^T T u) is parallel.
// (D_i, D_{i-1}) and (E_i, E_{i+1}) are rescaled together by a power of two
// every 4 rows, which leaves the pivots unchanged. Warps 2.. sum the symbol
// trace over the pixels [pix0, pix1) meanwhile (projected mode); all
// threads call it (at least 96). wk: 3 kk doubles.
__device__ double sel_eval_tw(const GcvSelectArgs& a, int kk, const double* dg, const double* eo, const double* f,
                              double r02, double gamma, double* u, double* wk, double* sh, double* tr_out, int pix0,
                              int pix1) {
  double* X0 = wk;            // b_i; minor D_i / E_i; 1 / pivot_i
  double* X1 = wk + kk;       // a^2 of the recurrence; previous minor; multiplier l_i (i < m) / r_i (i > m)
  double* X2 = wk + 2 * kk;   // eliminated right-hand side; then its product with 1 / pivot_i
  const double g1 = 1.0 - gamma, g0 = gamma;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int m = kk >> 1;
  __shared__ double s_trp[32];
  __shared__ double s_tw[2];
  // (0) coefficients
  for (int i = tid; i < kk; i += blockDim.x) {
    X0[i] = fma(g1, dg[i], g0);
    double c = 0.0;
    if (i < m && i > 0) c = g1 * eo[i - 1];
    else if (i > m && i + 1 < kk) c = g1 * eo[i];
    X1[i] = c * c;
  }
  __syncthreads();
  // (1) leading minors (thread 0) || trailing minors (thread 32) || trace partial sums (warps 2..)
  if (tid == 0) {
    double dm1 = 1.0, dm2 = 0.0;
    for (int i = 0; i < m; ++i) {
      const double di = fma(-X1[i], dm2, X0[i] * dm1);
      X0[i] = di;
      X1[i] = dm1;
      dm2 = dm1;
      dm1 = di;
      if ((i & 3) == 3 && di != 0.0) {
        const double sc = exp2_neg_exponent(di);
        dm1 *= sc;
        dm2 *= sc;
      }
    }
  } else if (tid == 32) {
    double em1 = 1.0, em2 = 0.0;
    for (int i = kk - 1, c = 0; i > m; --i, ++c) {
      const double ei = fma(-X1[i], em2, X0[i] * em1);
      X0[i] = ei;
      X1[i] = em1;
      em2 = em1;
      em1 = ei;
      if ((c & 3) == 3 && ei != 0.0) {
        const double sc = exp2_neg_exponent(ei);
        em1 *= sc;
        em2 *= sc;
      }
    }
  } else if (wid >= 2) {
    const float gs = (float)(gamma * a.s);
    float sum = 0.f, comp = 0.f;
    constexpr int B = 8;
    const int nt = blockDim.x - 64;
    for (int base = pix0 + tid - 64; base < pix1; base += nt * B) {
      float r[B];
#pragma unroll
      for (int q = 0; q < B; ++q) {
        const int i = base + q * nt;
        r[q] = i < pix1 ? __ldg(a.rho + i) : -1.f;
      }
#pragma unroll
      for (int q = 0; q < B; ++q) {
        if (r[q] < 0.f) continue;
        const float term = __frcp_rn(1.0f + gs * r[q]);
        const float y = term - comp;
        const float t = sum + y;
        comp = (t - sum) - y;
        sum = t;
      }
    }
    double trp = warp_sum((double)sum - (double)comp);
    if (lane == 0) s_trp[wid] = trp;
  }
  __syncthreads();
  // (2) reciprocals of the pivots and the multipliers, in parallel
  for (int i = tid; i < kk; i += blockDim.x) {
    if (i == m) continue;
    const double d = X0[i];
    const double inv = d != 0.0 ? X1[i] * rcp_d(d) : 0.0;
    X0[i] = inv;
    X1[i] = (i < m ? g1 * eo[i] : g1 * eo[i - 1]) * inv;
  }
  __syncthreads();
  // (3) eliminated right-hand sides, downwards (thread 0) and upwards
  //     (thread 32); trace total (warp 2)
  if (tid == 0) {
    if (m > 0) {
      double y = f[0];
      X2[0] = y;
      for (int i = 1; i < m; ++i) {
        y = fma(-X1[i - 1], y, f[i]);
        X2[i] = y;
      }
      s_tw[0] = X1[m - 1] * y;
    } else {
      s_tw[0] = 0.0;
    }
  } else if (tid == 32) {
    if (m + 1 < kk) {
      double z = f[kk - 1];
      X2[kk - 1] = z;
      for (int i = kk - 2; i > m; --i) {
        z = fma(-X1[i + 1], z, f[i]);
        X2[i] = z;
      }
      s_tw[1] = X1[m + 1] * z;
    } else {
      s_tw[1] = 0.0;
    }
  } else if (wid == 2) {
    const int nw = blockDim.x >> 5;
    double t = (lane >= 2 && lane < nw) ? s_trp[lane] : 0.0;
    t = warp_sum(t);
    if (lane == 0) *tr_out = t;
  }
  __syncthreads();
  // (3b) the twisted row m; the other rows' eliminated right-hand sides
  //      times 1 / pivot
  for (int i = tid; i < kk; i += blockDim.x) {
    if (i != m) {
      X2[i] *= X0[i];
    } else {
      double gm = X0[m];
      if (m > 0) gm -= (g1 * eo[m - 1]) * X1[m - 1];
      if (m + 1 < kk) gm -= (g1 * eo[m]) * X1[m + 1];
      u[m] = (f[m] - s_tw[0] - s_tw[1]) * rcp_d(gm);
    }
  }
  __syncthreads();
  // (3c) back substitution outwards from row m
  if (tid == 0) {
    double un = u[m];
    for (int i = m - 1; i >= 0; --i) {
      un = fma(-X1[i], un, X2[i]);
      u[i] = un;
    }
  } else if (tid == 32) {
    double un = u[m];
    for (int i = m + 1; i < kk; ++i) {
      un = fma(-X1[i], un, X2[i]);
      u[i] = un;
    }
  }
  __syncthreads();
  // (4) u^T T u
  double q[1] = {0.0};
  for (int i = tid; i < kk; i += blockDim.x) {
    double tu = dg[i] * u[i];
    if (i > 0) tu += eo[i - 1] * u[i - 1];
    if (i + 1 < kk) tu += eo[i] * u[i + 1];
    q[0] += u[i] * tu;
  }
  sel_sumN<1>(q, kk, sh);
  return gamma * gamma * q[0] + r02;
}

// Numerator gamma^2 u^T T u + r0^2 for one gamma by one warp (the grid
// points of the cluster selector): the twisted elimination of sel_eval_tw,
// its two recurrences in lanes 0 and 1, which run them as one instruction
// stream (an FP64 warp instruction costs the same for one lane or two), and
// its parallel phases over the lanes. X: 4 kk doubles of scratch (global);
// the whole warp calls it; the result is in every lane.
__device__ double sel_numerator_warp(int kk, const double* dg, const double* eo, const double* f, double r02,
                                     double gamma, double* X) {
  double* X0 = X;
  double* X1 = X + kk;
  double* X2 = X + 2 * kk;
  double* u = X + 3 * kk;
  const double g1 = 1.0 - gamma, g0 = gamma;
  const int lane = threadIdx.x & 31;
  const int m = kk >> 1;
  const bool fwd = lane == 0;
  for (int i = lane; i < kk; i += 32) {
    X0[i] = fma(g1, dg[i], g0);
    double c = 0.0;
    if (i < m && i > 0) c = g1 * eo[i - 1];
    else if (i > m && i + 1 < kk) c = g1 * eo[i];
    X1[i] = c * c;
  }
  __syncwarp();
  // minors: leading (lane 0, rows 0..m-1), trailing (lane 1, rows kk-1..m+1)
  if (lane < 2) {
    const int ns = fwd ? m : kk - 1 - m;
    double p1 = 1.0, p2 = 0.0;
    for (int st = 0; st < ns; ++st) {
      const int i = fwd ? st : kk - 1 - st;
      const double di = fma(-X1[i], p2, X0[i] * p1);
      X0[i] = di;
      X1[i] = p1;
      p2 = p1;
      p1 = di;
      if ((st & 3) == 3 && di != 0.0) {
        const double sc = exp2_neg_exponent(di);
        p1 *= sc;
        p2 *= sc;
      }
    }
  }
  __syncwarp();
  for (int i = lane; i < kk; i += 32) {
    if (i == m) continue;
    const double d = X0[i];
    const double inv = d != 0.0 ? X1[i] * rcp_d(d) : 0.0;
    X0[i] = inv;
    X1[i] = (i < m ? g1 * eo[i] : g1 * eo[i - 1]) * inv;
  }
  __syncwarp();
  // eliminated right-hand sides: downwards (lane 0), upwards (lane 1)
  double tw = 0.0;
  if (lane < 2 && (fwd ? m > 0 : m + 1 < kk)) {
    const int ns = fwd ? m - 1 : kk - 2 - m;
    double y = fwd ? f[0] : f[kk - 1];
    X2[fwd ? 0 : kk - 1] = y;
    for (int st = 0; st < ns; ++st) {
      const int i = fwd ? 1 + st : kk - 2 - st;
      y = fma(-X1[fwd ? i - 1 : i + 1], y, f[i]);
      X2[i] = y;
    }
    tw = X1[fwd ? m - 1 : m + 1] * y;
  }
  const double tw0 = __shfl_sync(0xffffffffu, tw, 0), tw1 = __shfl_sync(0xffffffffu, tw, 1);
  __syncwarp();
  for (int i = lane; i < kk; i += 32) {
    if (i != m) {
      X2[i] *= X0[i];
    } else {
      double gm = X0[m];
      if (m > 0) gm -= (g1 * eo[m - 1]) * X1[m - 1];
      if (m + 1 < kk) gm -= (g1 * eo[m]) * X1[m + 1];
      u[m] = (f[m] - tw0 - tw1) * rcp_d(gm);
    }
  }
  __syncwarp();
  // back substitution outwards: lane 0 rows m-1..0, lane 1 rows m+1..kk-1
  if (lane < 2) {
    const int ns = fwd ? m : kk - 1 - m;
    double un = u[m];
    for (int st = 0; st < ns; ++st) {
      const int i = fwd ? m - 1 - st : m + 1 + st;
      un = fma(-X1[i], un, X2[i]);
      u[i] = un;
    }
  }
  __syncwarp();
  double q = 0.0;
  for (int i = lane; i < kk; i += 32) {
    double tu = dg[i] * u[i];
    if (i > 0) tu += eo[i - 1] * u[i - 1];
    if (i + 1 < kk) tu += eo[i] * u[i + 1];
    q += u[i] * tu;
  }
  q = warp_sum(q);
  return gamma * gamma * q + r02;
}

// Symbol trace sum_i 1 / (1 + gamma s rho_i) over the pixels [pix0, pix1)
// for one gamma (all threads; loads in batches of 8 per thread,
// Kahan-compensated float sums).
__device__ double sel_trace_one(const GcvSelectArgs& a, double gamma, double* sh, int pix0, int pix1) {
  const float gs = (float)(gamma * a.s);
  float sum = 0.f, comp = 0.f;
  constexpr int B = 8;
  for (int base = pix0 + threadIdx.x; base < pix1; base += blockDim.x * B) {
    float r[B];
#pragma unroll
    for (int q = 0; q < B; ++q) {
      const int i = base + q * blockDim.x;
      r[q] = i < pix1 ? __ldg(a.rho + i) : -1.f;
    }
#pragma unroll
    for (int q = 0; q < B; ++q) {
      if (r[q] < 0.f) continue;
      const float term = __frcp_rn(1.0f + gs * r[q]);
      const float y = term - comp;
      const float t = sum + y;
      comp = (t - sum) - y;
      sum = t;
    }
  }
  return sel_block_sum((double)sum - (double)comp, sh);
}

// Trace term for a set of gammas (all threads); returns per-gamma traces in
// tr[] (projected mode: over the pixels [pix0, pix1)).
__device__ void sel_traces(const GcvSelectArgs& a, const double* lam, int ng, const double* gam, double* tr,
                           double* sh, int pix0, int pix1) {
  for (int g = 0; g < ng; ++g) {
    if (a.exact) {
      double part = 0.0;
      for (int j = threadIdx.x; j < a.kk; j += blockDim.x) {
        const double l = lam[j];
        part += l / (l + gam[g] * (1.0 - l));
      }
      const double t = sel_block_sum(part, sh);
      if (threadIdx.x == 0) tr[g] = t;
    } else {
      const double t = sel_trace_one(a, gam[g], sh, pix0, pix1);
      if (threadIdx.x == 0) tr[g] = t;
    }
  }
  __syncthreads();
}

// Symbol traces on the first selection grid (npts log-spaced gammas on
// [lo, hi], the same points as k_gcv_select) in one pass over rho by many
// blocks: each block takes a chunk of pixels into shared memory and every
// thread sums its gammas over the chunk (Kahan); block partials as (hi, lo)
// float pairs, combined in a fixed order by the last block.
constexpr int TRT_CHUNK = 4096;
__global__ void __launch_bounds__(256) k_trace_table(const float* __restrict__ rho, int npix, double s, double lo,
                                                     double hi, int npts, float2* part, unsigned* cnt,
                                                     double* tab) {
  __shared__ float sr[TRT_CHUNK];
  __shared__ int s_last;
  const int nb = gridDim.x;
  const double step = (hi - lo) / (npts - 1);
  float sum[SEL_MAXPTS / 32 + 1], comp[SEL_MAXPTS / 32 + 1];
  float gs[SEL_MAXPTS / 32 + 1];
  constexpr int G = SEL_MAXPTS / 32 + 1;
  // thread t handles gammas t % 32 + 32 q (lanes of a warp cover the gammas;
  // warps split the chunk)
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int q = 0; q < G; ++q) {
    sum[q] = comp[q] = 0.f;
    const int j = lane + 32 * q;
    gs[q] = j < npts ? (float)(pow(10.0, (j == npts - 1) ? hi : lo + j * step) * s) : 0.f;
  }
  for (int ch = blockIdx.x; ch * TRT_CHUNK < npix; ch += nb) {
    const int beg = ch * TRT_CHUNK;
    const int len = min(TRT_CHUNK, npix - beg);
    __syncthreads();
    for (int i = threadIdx.x; i < len; i += blockDim.x) sr[i] = rho[beg + i];
    __syncthreads();
    for (int i = wid; i < len; i += nw) {
      const float r = sr[i];
#pragma unroll
      for (int q = 0; q < G; ++q) {
        const float term = __frcp_rn(1.0f + gs[q] * r);
        const float y = term - comp[q];
        const float t = sum[q] + y;
        comp[q] = (t - sum[q]) - y;
        sum[q] = t;
      }
    }
  }
  // per-gamma block partial: combine the warps' (sum, -comp) pairs
  __shared__ float2 sw[8][SEL_MAXPTS + 32];
#pragma unroll
  for (int q = 0; q < G; ++q) sw[wid][lane + 32 * q] = make_float2(sum[q], -comp[q]);
  __syncthreads();
  for (int j = threadIdx.x; j < npts; j += blockDim.x) {
    float h = 0.f, l = 0.f;
    for (int w = 0; w < nw; ++w) df_add(h, l, sw[w][j].x, sw[w][j].y);
    part[(size_t)j * nb + blockIdx.x] = make_float2(h, l);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    s_last = (atomicAdd(cnt, 1u) == (unsigned)nb - 1);
    __threadfence();
  }
  __syncthreads();
  if (!s_last) return;
  for (int j = threadIdx.x; j < npts; j += blockDim.x) {
    float h = 0.f, l = 0.f;
    df_sum_loads(part + (size_t)j * nb, nb, h, l);
    tab[j] = (double)h + (double)l;
  }
  if (threadIdx.x == 0) *cnt = 0;
}

// Up to three independent selections (different basis dimensions of one GCV
// call) in one launch, one block each.
__global__ void __launch_bounds__(SEL_THREADS) k_gcv_select(GcvSelectArgs a0, GcvSelectArgs a1, GcvSelectArgs a2) {
  GcvSelectArgs a = a0;
  if (blockIdx.x == 1) a = a1;
  else if (blockIdx.x == 2) a = a2;
  extern __shared__ __align__(16) double sdyn[];
  __shared__ double sh[32 * 3];
  __shared__ double s_gam[SEL_MAXPTS], s_tr[SEL_MAXPTS], s_f[SEL_MAXPTS];
  __shared__ double s_bc[4];
  const int kk = a.kk, ld = a.ld, tid = threadIdx.x, nth = blockDim.x;
  const int lds = sel_lds(kk);
  const bool in_smem = kk <= SEL_SMEM_K;
  double* pA = sdyn;
  double* pD = pA + kk;
  double* dg = pD + kk;               // tridiagonal diagonal
  double* eo = dg + kk;               // tridiagonal off-diagonal
  double* u = eo + kk;
  double* p = u + kk;
  double* colc = p + kk;
  double* rdiag = colc + kk;
  double* fvec = rdiag + kk;
  double* lam = fvec + kk;            // eigenvalues of T (exact mode)
  double* S = in_smem ? sdyn + SEL_NVEC * kk : a.work;          // working matrix, pitch lds
  double* X = in_smem ? a.work : a.work + (size_t)kk * lds;     // R^{-1} G_A (global)
  double* Cg = X + (size_t)kk * kk;                             // R^{-1} G_A R^{-T} (global)
  double* scratch = Cg + (size_t)kk * kk;                       // grid Thomas scratch, 2 kk per point
  auto mapk = [&](int i) { return (a.kshift >= 0 && i == kk - 1) ? a.kshift : i; };
  auto GAe = [&](int i, int j) {
    i = mapk(i); j = mapk(j);
    return i <= j ? a.GA[(size_t)i * ld + j] : a.GA[(size_t)j * ld + i];
  };
  auto GDe = [&](int i, int j) {
    i = mapk(i); j = mapk(j);
    return i <= j ? a.GD[(size_t)i * ld + j] : a.GD[(size_t)j * ld + i];
  };
  // 1. S = M = G_A + G_D (lower triangle), p_A = g_A, p_D = g_D
  // (element loops run one row per warp, lanes over the columns: no integer
  // division per element)
  const int lane = tid & 31, wid = tid >> 5, nwarp = nth >> 5;
  for (int i = wid; i < kk; i += nwarp)
    for (int j = lane; j <= i; j += 32) S[i * lds + j] = GAe(i, j) + GDe(i, j);
  for (int i = tid; i < kk; i += nth) { pA[i] = a.gA[mapk(i)]; pD[i] = a.gD[mapk(i)]; }
  __syncthreads();
  if (tid == 0) {
    double md = 0.0;
    for (int i = 0; i < kk; ++i) md = fmax(md, S[i * lds + i]);
    s_bc[0] = md;
  }
  __syncthreads();
  const double piv_floor = 1e-14 * s_bc[0];
  // 2. Cholesky M = R R^T (lower, in place); rdiag = 1 / diag(R)
  for (int c = 0; c < kk; ++c) {
    if (tid == 0) {
      const double piv = S[c * lds + c];
      const double pv = piv > piv_floor ? piv : piv_floor;
      const double ir = rsqrt_d(pv);
      S[c * lds + c] = pv * ir;
      rdiag[c] = ir;
    }
    __syncthreads();
    const double ir = rdiag[c];
    for (int i = c + 1 + tid; i < kk; i += nth) {
      const double v = S[i * lds + c] * ir;
      S[i * lds + c] = v;
      colc[i] = v;
    }
    __syncthreads();
    for (int i = c + 1 + wid; i < kk; i += nwarp) {
      const double ci = colc[i];
      double* Si = S + (size_t)i * lds;
      for (int j = c + 1 + lane; j <= i; j += 32) Si[j] -= ci * colc[j];
    }
    __syncthreads();
  }
  // 3. X = R^{-1} G_A, p_A <- R^{-1} p_A, p_D <- R^{-1} p_D (one column per
  //    thread, eight partial sums to shorten the dependent chain)
  for (int q = tid; q < kk + 2; q += nth) {
    double* vcol = q == kk ? pA : pD;
    for (int i = 0; i < kk; ++i) {
      double sacc[8];
      sacc[0] = q < kk ? GAe(i, q) : vcol[i];
#pragma unroll
      for (int r = 1; r < 8; ++r) sacc[r] = 0.0;
      const double* Ri = S + (size_t)i * lds;
      int l = 0;
      if (q < kk) {
        for (; l + 7 < i; l += 8) {
#pragma unroll
          for (int r = 0; r < 8; ++r) sacc[r] -= Ri[l + r] * X[(size_t)(l + r) * kk + q];
        }
        for (; l < i; ++l) sacc[0] -= Ri[l] * X[(size_t)l * kk + q];
      } else {
        for (; l + 7 < i; l += 8) {
#pragma unroll
          for (int r = 0; r < 8; ++r) sacc[r] -= Ri[l + r] * vcol[l + r];
        }
        for (; l < i; ++l) sacc[0] -= Ri[l] * vcol[l];
      }
      const double v = (((sacc[0] + sacc[1]) + (sacc[2] + sacc[3])) + ((sacc[4] + sacc[5]) + (sacc[6] + sacc[7]))) *
                       rdiag[i];
      if (q < kk) X[(size_t)i * kk + q] = v; else vcol[i] = v;
    }
  }
  __syncthreads();
  // 4. C = R^{-1} X^T (= R^{-1} G_A R^{-T}), column q per thread
  for (int q = tid; q < kk; q += nth) {
    for (int i = 0; i < kk; ++i) {
      double sacc[8];
      sacc[0] = X[(size_t)q * kk + i];
#pragma unroll
      for (int r = 1; r < 8; ++r) sacc[r] = 0.0;
      const double* Ri = S + (size_t)i * lds;
      int l = 0;
      for (; l + 7 < i; l += 8) {
#pragma unroll
        for (int r = 0; r < 8; ++r) sacc[r] -= Ri[l + r] * Cg[(size_t)(l + r) * kk + q];
      }
      for (; l < i; ++l) sacc[0] -= Ri[l] * Cg[(size_t)l * kk + q];
      Cg[(size_t)i * kk + q] =
          (((sacc[0] + sacc[1]) + (sacc[2] + sacc[3])) + ((sacc[4] + sacc[5]) + (sacc[6] + sacc[7]))) * rdiag[i];
    }
  }
  __syncthreads();
  // 5. S = symmetrised C (lower triangle; R is no longer needed)
  for (int i = wid; i < kk; i += nwarp)
    for (int j = lane; j <= i; j += 32) S[i * lds + j] = 0.5 * (Cg[(size_t)i * kk + j] + Cg[(size_t)j * kk + i]);
  __syncthreads();
  // 6. Householder tridiagonalisation C = Q T Q^T on the lower triangle;
  //    p_A, p_D <- Q^T p_A, Q^T p_D.
  for (int k = 0; k + 2 < kk; ++k) {
    const int len = kk - k - 1;
    double nx[1] = {0.0};
    for (int i = tid; i < len; i += nth) {
      const double xv = S[(k + 1 + i) * lds + k];
      u[i] = xv;
      nx[0] += xv * xv;
    }
    sel_sumN<1>(nx, len, sh);
    const double nx2 = nx[0];
    const double x0 = u[0];
    if (nx2 - x0 * x0 <= 1e-300 * (1.0 + nx2)) continue;   // column already reduced (uniform)
    if (tid == 0) {
      const double inx = rsqrt_d(nx2);
      const double nrm = nx2 * inx;
      const double alpha = x0 >= 0 ? -nrm : nrm;
      s_bc[1] = alpha;
      s_bc[2] = rsqrt_d(2.0 * nrm * (nrm + fabs(x0)));
    }
    __syncthreads();
    const double alpha = s_bc[1], inv_nu = s_bc[2];
    for (int i = tid; i < len; i += nth) u[i] = (u[i] - (i == 0 ? alpha : 0.0)) * inv_nu;
    __syncthreads();
    // p = C' u with C' the trailing block (lower storage: row part, then column part)
    const double* Sb = S + (size_t)(k + 1) * lds + (k + 1);
    for (int i = tid; i < len; i += nth) {
      double s4[4] = {0.0, 0.0, 0.0, 0.0};
      const double* row = Sb + (size_t)i * lds;
      int j = 0;
      for (; j + 3 < i; j += 4) {
#pragma unroll
        for (int r = 0; r < 4; ++r) s4[r] += row[j + r] * u[j + r];
      }
      for (; j < i; ++j) s4[0] += row[j] * u[j];
      j = i;
      for (; j + 3 < len; j += 4) {
#pragma unroll
        for (int r = 0; r < 4; ++r) s4[r] += Sb[(size_t)(j + r) * lds + i] * u[j + r];
      }
      for (; j < len; ++j) s4[0] += Sb[(size_t)j * lds + i] * u[j];
      p[i] = (s4[0] + s4[1]) + (s4[2] + s4[3]);
    }
    __syncthreads();
    double kd[3] = {0.0, 0.0, 0.0};
    for (int i = tid; i < len; i += nth) {
      kd[0] += u[i] * p[i];
      kd[1] += u[i] * pA[k + 1 + i];
      kd[2] += u[i] * pD[k + 1 + i];
    }
    sel_sumN<3>(kd, len, sh);
    const double K = kd[0], da = kd[1], dd = kd[2];
    for (int i = tid; i < len; i += nth) p[i] = 2.0 * p[i] - 2.0 * K * u[i];   // w
    __syncthreads();
    for (int ii = wid; ii < len; ii += nwarp) {
      const double ui = u[ii], wi = p[ii];
      double* Si = S + (size_t)(k + 1 + ii) * lds + (k + 1);
      for (int jj = lane; jj <= ii; jj += 32) Si[jj] -= ui * p[jj] + wi * u[jj];
    }
    for (int i = tid; i < len; i += nth) {
      pA[k + 1 + i] -= 2.0 * da * u[i];
      pD[k + 1 + i] -= 2.0 * dd * u[i];
    }
    if (tid == 0) S[(size_t)(k + 1) * lds + k] = alpha;
    __syncthreads();
  }
  for (int i = tid; i < kk; i += nth) {
    dg[i] = S[(size_t)i * lds + i];
    eo[i] = (i + 1 < kk) ? S[(size_t)(i + 1) * lds + i] : 0.0;
  }
  __syncthreads();
  // 6b. w0 = T^{-1} p_A, f = p_A + p_D - w0, r0^2 = ||b||^2 - p_A . w0.
  //     One Thomas sweep: T can be numerically singular (exact mode on a tiny
  //     level), where sequential elimination stays accurate and parallel
  //     cyclic reduction does not.
  if (tid == 0) {
    sel_tri_solve(kk, dg, eo, pA, 0.0, p, u, 0.0);
    double pw = 0.0;
    for (int i = 0; i < kk; ++i) {
      pw += pA[i] * u[i];
      fvec[i] = pA[i] + pD[i] - u[i];
    }
    s_bc[3] = pw;
  }
  __syncthreads();
  const double r02 = (a.bnorm2 - s_bc[3]) > 0.0 ? (a.bnorm2 - s_bc[3]) : 0.0;
  // 7. exact mode: eigenvalues of T by bisection (Sturm counts), one per thread
  if (a.exact) {
    double glo = 0.0, ghi = 0.0;
    for (int i = 0; i < kk; ++i) {   // Gershgorin interval
      const double r = (i > 0 ? fabs(eo[i - 1]) : 0.0) + (i + 1 < kk ? fabs(eo[i]) : 0.0);
      glo = fmin(glo, dg[i] - r);
      ghi = fmax(ghi, dg[i] + r);
    }
    for (int j = tid; j < kk; j += nth) {
      double l = glo, h = ghi;
      for (int it = 0; it < 64; ++it) {
        const double x = 0.5 * (l + h);
        int cnt = 0;
        double q = dg[0] - x;
        if (q < 0) ++cnt;
        for (int i = 1; i < kk; ++i) {
          const double qq = (q != 0.0) ? q : 1e-300;
          q = dg[i] - x - eo[i - 1] * eo[i - 1] / qq;
          if (q < 0) ++cnt;
        }
        if (cnt > j) h = x; else l = x;   // cnt = number of eigenvalues below x
      }
      double v = 0.5 * (l + h);
      lam[j] = v < 0.0 ? 0.0 : (v > 1.0 ? 1.0 : v);
    }
    __syncthreads();
  }
  // 8. grid search (parallel over the grid points) with widening, then Brent
  const int npts = a.npts < SEL_MAXPTS ? a.npts : SEL_MAXPTS;
  double lo = a.lo, hi = a.hi;
  int ext = 0, jbest = 0;
  double fbest = 0.0, step = 0.0;
  for (;;) {
    step = (hi - lo) / (npts - 1);
    for (int j = tid; j < npts; j += nth) s_gam[j] = pow(10.0, (j == npts - 1) ? hi : lo + j * step);
    __syncthreads();
    if (ext == 0 && a.trace_tab && !a.exact) {
      for (int j = tid; j < npts; j += nth) s_tr[j] = a.trace_tab[j];
      __syncthreads();
    } else {
      sel_traces(a, lam, npts, s_gam, s_tr, sh, 0, a.npix);
    }
    for (int j = tid; j < npts; j += nth) {
      const double num = sel_numerator(kk, dg, eo, fvec, r02, s_gam[j], scratch + (size_t)j * 2 * kk,
                                       scratch + (size_t)j * 2 * kk + kk);
      const double den = a.n - s_tr[j];
      s_f[j] = num / (den * den);
    }
    __syncthreads();
    jbest = 0;
    fbest = s_f[0];
    for (int j = 1; j < npts; ++j)
      if (s_f[j] < fbest) { fbest = s_f[j]; jbest = j; }
    __syncthreads();
    if (jbest == 0 && ext < a.max_ext) { lo -= 4.0; ++ext; continue; }
    if (jbest == npts - 1 && ext < a.max_ext) { hi += 4.0; ++ext; continue; }
    break;
  }
  auto tgrid = [&](int j) { return (j == npts - 1) ? hi : lo + j * step; };
  // S is free once T is extracted: scratch of the trial-gamma solves
  auto feval = [&](double t) -> double {
    const double gam = pow(10.0, t);
    const double num = sel_eval_seq(a, kk, dg, eo, fvec, r02, lam, gam, u, S, sh, &s_bc[2]);
    const double den = a.n - s_bc[2];
    __syncthreads();
    return num / (den * den);
  };
  double A = tgrid(jbest > 0 ? jbest - 1 : 0);
  double B = tgrid(jbest < npts - 1 ? jbest + 1 : npts - 1);
  // Brent (golden section + parabolic interpolation); every thread runs the
  // same control flow on the same values.
  const double cgold = 0.5 * (3.0 - sqrt(5.0));
  const double sqeps = sqrt(2.220446049250313e-16);
  double x = A + cgold * (B - A), w = x, v = x;
  double fx = feval(x), fw = fx, fv = fx;
  double d = 0.0, e = 0.0;
  for (int nfev = 1; nfev < 500; ++nfev) {
    const double xm = 0.5 * (A + B);
    const double tol1 = sqeps * fabs(x) + a.tolx / 3.0;
    const double tol2 = 2.0 * tol1;
    if (fabs(x - xm) <= tol2 - 0.5 * (B - A)) break;
    bool golden = true;
    if (fabs(e) > tol1) {
      double r = (x - w) * (fx - fv);
      double q = (x - v) * (fx - fw);
      double pp = (x - v) * q - (x - w) * r;
      q = 2.0 * (q - r);
      if (q > 0.0) pp = -pp;
      q = fabs(q);
      const double etemp = e;
      e = d;
      if (fabs(pp) < fabs(0.5 * q * etemp) && pp > q * (A - x) && pp < q * (B - x)) {
        d = pp / q;
        const double uu = x + d;
        if ((uu - A) < tol2 || (B - uu) < tol2) d = (xm >= x) ? tol1 : -tol1;
        golden = false;
      }
    }
    if (golden) { e = (x < xm) ? (B - x) : (A - x); d = cgold * e; }
    const double uu = (fabs(d) >= tol1) ? x + d : x + (d > 0 ? tol1 : -tol1);
    const double fu = feval(uu);
    if (fu <= fx) {
      if (uu < x) B = x; else A = x;
      v = w; fv = fw; w = x; fw = fx; x = uu; fx = fu;
    } else {
      if (uu < x) A = uu; else B = uu;
      if (fu <= fw || w == x) { v = w; fv = fw; w = uu; fw = fu; }
      else if (fu <= fv || v == x || v == w) { v = uu; fv = fu; }
    }
  }
  const double tbest = (fx <= fbest) ? x : tgrid(jbest);
  if (tid == 0) {
    a.out[0] = pow(10.0, tbest);
    a.out[1] = (double)ext;
    a.out[2] = (fx <= fbest) ? fx : fbest;
  }
}

// ---- the selection on a thread-block cluster ---------------------------------
// The same computation as k_gcv_select for one projected-mode selection,
// spread over a cluster of SCL_NC CTAs (one per SM), since one SM issues only
// about two FP64 FMAs per clock. Row i of the working matrices belongs to
// CTA i % SCL_NC.
//  * Cholesky, right-looking: per column, every CTA sends its rows' entries
//    to all CTAs (distributed shared memory), and every CTA forms the same
//    column of R and updates its own rows; so every CTA ends with a full
//    copy of R (packed lower triangle). The next column's entries are
//    updated and sent first, so the barrier completes during the rest of
//    the update.
//  * X = R^{-1} [G_A | g_A | g_D] and C = R^{-1} X^T: each CTA solves its own
//    columns (right-looking over the rows of R, its local copy), X passing
//    through global memory between the two; column q of C is row q, so each
//    CTA ends with its own rows of C (full rows).
//  * Householder: one exchange per step carries the per-CTA partials of
//    C u (summed in CTA order) and row k+1 from its owner; every CTA then
//    forms the same w, K, the next column (row k+1 after the update, by
//    symmetry) and the next reflector, and updates its own rows.
//  * T's diagonals are gathered; w0 and the Brent control flow run in every
//    CTA on the same values, while the symbol traces (split by pixel range)
//    and the grid numerators (split by point) are computed once and
//    exchanged. Each Brent evaluation uses the twisted elimination.
// Every value that more than one CTA computes is computed from the same data
// in the same order, so the copies agree bit for bit.
constexpr int SCL_NC = 8;
constexpr int SCL_THREADS = 256;
constexpr int SCL_MAXK = 164;

struct SclLayout {
  int K, nrl, ncl;
  size_t rp, mr, xc, vec, cb, pb, total;   // offsets in doubles
};
__host__ __device__ inline SclLayout scl_layout(int K) {
  SclLayout L;
  L.K = K;
  L.nrl = (K + SCL_NC - 1) / SCL_NC;
  L.ncl = (K + 2 + SCL_NC - 1) / SCL_NC;
  L.rp = 0;
  L.mr = L.rp + (size_t)K * (K + 1) / 2;
  L.xc = L.mr + (size_t)L.nrl * K;
  L.vec = L.xc + (size_t)K * L.ncl;
  L.cb = L.vec + (size_t)12 * K;
  L.pb = L.cb + (size_t)2 * K;
  L.total = L.pb + (size_t)2 * SCL_NC * K;
  return L;
}
__host__ __device__ inline size_t rp_at(int i, int j) { return (size_t)i * (i + 1) / 2 + j; }

// In-place forward substitution R x = rhs on nc columns held as
// Xc[i * nc + c] (R from the packed copy, rdiag = 1 / diag R), right-looking
// over the rows so every step is parallel over (row, column).
__device__ void scl_forward(int K, int nc, const double* Rp, const double* rdiag, double* Xc) {
  const int tid = threadIdx.x, nth = blockDim.x;
  for (int i = 0; i < K; ++i) {
    if (tid < nc) Xc[(size_t)i * nc + tid] *= rdiag[i];
    __syncthreads();
    const int rows = K - i - 1;
    for (int idx = tid; idx < rows * nc; idx += nth) {
      const int i2 = i + 1 + idx / nc, c = idx - (idx / nc) * nc;
      Xc[(size_t)i2 * nc + c] -= Rp[rp_at(i2, i)] * Xc[(size_t)i * nc + c];
    }
    __syncthreads();
  }
}

// Split cluster barrier (every thread of every CTA of the cluster, in
// arrive / wait alternation): arrive releases this thread's earlier writes,
// including those to other CTAs' shared memory; wait returns once every
// thread of the cluster has arrived and acquires their writes.
__device__ __forceinline__ void scl_arrive() { asm volatile("barrier.cluster.arrive.release.aligned;\n" ::: "memory"); }
__device__ __forceinline__ void scl_wait() { asm volatile("barrier.cluster.wait.acquire.aligned;\n" ::: "memory"); }

// Householder step arithmetic with explicit roundings, so that every CTA
// that evaluates an entry gets the same bits: w_j = 2 p_j - 2 K u_j and the
// rank-2 update m - (u_i w_j + w_i u_j).
__device__ __forceinline__ double hh_w(double m2K, double uj, double pj) { return __fma_rn(m2K, uj, 2.0 * pj); }
__device__ __forceinline__ double hh_upd(double m, double ui, double wj, double wi, double uj) {
  return __dsub_rn(m, __fma_rn(ui, wj, __dmul_rn(wi, uj)));
}

// Reflector of the column x (len entries) by one warp: alpha = -sign(x_0)
// ||x||, u = (x - alpha e_0) / sqrt(2 ||x|| (||x|| + |x_0|)), so that
// (I - 2 u u^T) x = alpha e_0; a column already reduced gives u = 0 and
// alpha = x_0 (the step leaves the matrix as it is).
__device__ void scl_reflector_warp(int len, const double* x, double* u, double* alpha_out) {
  const int lane = threadIdx.x & 31;
  double acc = 0.0;
  for (int j = lane; j < len; j += 32) acc += x[j] * x[j];
  const double nx2 = warp_sum(acc);
  const double x0 = x[0];
  const bool reduced = nx2 - x0 * x0 <= 1e-300 * (1.0 + nx2);
  double alpha = x0, inv_nu = 0.0;
  if (!reduced) {
    const double nrm = nx2 * rsqrt_d(nx2);
    alpha = x0 >= 0 ? -nrm : nrm;
    inv_nu = rsqrt_d(2.0 * nrm * (nrm + fabs(x0)));
  }
  for (int j = lane; j < len; j += 32) u[j] = reduced ? 0.0 : (x[j] - (j == 0 ? alpha : 0.0)) * inv_nu;
  if (lane == 0) *alpha_out = alpha;
}

// One selection on the calling cluster (every thread of its SCL_NC CTAs).
__device__ void sel_cl_run(const GcvSelectArgs& a) {
  namespace cg = cooperative_groups;
  cg::cluster_group cl = cg::this_cluster();
  extern __shared__ __align__(16) double sdyn[];
  __shared__ double sh[32 * 3];
  __shared__ double s_gam[SEL_MAXPTS], s_tr[SEL_MAXPTS], s_f[SEL_MAXPTS];
  __shared__ double s_bc[4];
  const int rank = (int)cl.block_rank();
  const int K = a.kk, ld = a.ld, tid = threadIdx.x, nth = blockDim.x;
  const int lane = tid & 31, wid = tid >> 5, nwarp = nth >> 5;
  const SclLayout Ly = scl_layout(K);
  const int nrl = Ly.nrl, ncl = Ly.ncl;
  double* Rp = sdyn + Ly.rp;
  double* Mr = sdyn + Ly.mr;      // own rows: M during Cholesky, then C
  double* Xc = sdyn + Ly.xc;      // own columns (X, then C)
  double* pA = sdyn + Ly.vec;
  double* pD = pA + K;
  double* dg = pD + K;
  double* eo = dg + K;
  double* u = eo + K;
  double* p = u + K;
  double* fvec = p + K;
  double* rdiag = fvec + K;
  double* colc = rdiag + K;
  double* wk3 = colc + K;         // 3 K, scratch of the trial-gamma solves
  double* cbuf = sdyn + Ly.cb;    // 2 K, double-buffered column exchange
  double* pbuf = sdyn + Ly.pb;    // 2 x SCL_NC x K partial products (double-buffered)
  double* Xg = a.work;            // K x K, X through global memory
  double* vg = Xg + (size_t)K * K;            // p_A, p_D through global memory (2 K)
  double* scratch = vg + 2 * (size_t)K;       // grid scratch, 4 K per point
  auto mapk = [&](int i) { return (a.kshift >= 0 && i == K - 1) ? a.kshift : i; };
  auto GAe = [&](int i, int j) {
    i = mapk(i); j = mapk(j);
    return i <= j ? a.GA[(size_t)i * ld + j] : a.GA[(size_t)j * ld + i];
  };
  auto GDe = [&](int i, int j) {
    i = mapk(i); j = mapk(j);
    return i <= j ? a.GD[(size_t)i * ld + j] : a.GD[(size_t)j * ld + i];
  };
  // 1. own rows of M = G_A + G_D (lower part); the pivot floor from the full diagonal
  for (int li = wid; li < nrl; li += nwarp) {
    const int i = rank + li * SCL_NC;
    if (i >= K) continue;
    for (int j = lane; j <= i; j += 32) Mr[(size_t)li * K + j] = GAe(i, j) + GDe(i, j);
  }
  if (tid == 0) {
    double md = 0.0;
    for (int i = 0; i < K; ++i) md = fmax(md, GAe(i, i) + GDe(i, i));
    s_bc[0] = md;
  }
  __syncthreads();
  const double piv_floor = 1e-14 * s_bc[0];
  cl.sync();   // every CTA of the cluster is running before the first remote store
  // 2. Cholesky M = R R^T, column by column. Each column's exchange is a
  //    split cluster barrier: a CTA updates its entries of the next column
  //    first, sends them and arrives, then updates the rest of its rows
  //    while the other CTAs catch up; it waits only before the next pivot.
  for (int idx = tid; idx < nrl * SCL_NC; idx += nth) {
    const int li = idx / SCL_NC, r = idx - li * SCL_NC;
    const int i = rank + li * SCL_NC;
    if (i < K) cl.map_shared_rank(cbuf, r)[i] = Mr[(size_t)li * K];
  }
  scl_arrive();
  for (int c = 0; c < K; ++c) {
    double* cb = cbuf + (size_t)(c & 1) * K;
    double* cbn = cbuf + (size_t)((c + 1) & 1) * K;
    scl_wait();
    if (tid == 0) {
      const double piv = cb[c];
      const double pv = piv > piv_floor ? piv : piv_floor;
      const double ir = rsqrt_d(pv);
      rdiag[c] = ir;
      Rp[rp_at(c, c)] = pv * ir;
    }
    __syncthreads();
    const double ir = rdiag[c];
    for (int i = c + 1 + tid; i < K; i += nth) {
      const double v = cb[i] * ir;
      Rp[rp_at(i, c)] = v;
      colc[i] = v;
    }
    __syncthreads();
    // own entries of column c+1, updated and sent
    if (c + 1 < K) {
      const double cn = colc[c + 1];
      for (int li = tid; li < nrl; li += nth) {
        const int i = rank + li * SCL_NC;
        if (i <= c || i >= K) continue;
        const double v = Mr[(size_t)li * K + c + 1] - colc[i] * cn;
        Mr[(size_t)li * K + c + 1] = v;
        for (int r = 0; r < SCL_NC; ++r) cl.map_shared_rank(cbn, r)[i] = v;
      }
    }
    scl_arrive();
    for (int li = wid; li < nrl; li += nwarp) {
      const int i = rank + li * SCL_NC;
      if (i <= c + 1 || i >= K) continue;
      const double ci = colc[i];
      double* Mi = Mr + (size_t)li * K;
      for (int j = c + 2 + lane; j <= i; j += 32) Mi[j] -= ci * colc[j];
    }
    __syncthreads();
  }
  scl_wait();
  // 3. X = R^{-1} [G_A | g_A | g_D], own columns q = rank + lq * SCL_NC
  for (int idx = tid; idx < K * ncl; idx += nth) {
    const int i = idx / ncl, lq = idx - (idx / ncl) * ncl;
    const int q = rank + lq * SCL_NC;
    double v = 0.0;
    if (q < K) v = GAe(i, q);
    else if (q == K) v = a.gA[mapk(i)];
    else if (q == K + 1) v = a.gD[mapk(i)];
    Xc[(size_t)i * ncl + lq] = v;
  }
  __syncthreads();
  scl_forward(K, ncl, Rp, rdiag, Xc);
  for (int idx = tid; idx < K * ncl; idx += nth) {
    const int i = idx / ncl, lq = idx - (idx / ncl) * ncl;
    const int q = rank + lq * SCL_NC;
    const double v = Xc[(size_t)i * ncl + lq];
    if (q < K) Xg[(size_t)i * K + q] = v;
    else if (q == K) vg[i] = v;
    else if (q == K + 1) vg[K + i] = v;
  }
  cl.sync();
  for (int i = tid; i < K; i += nth) { pA[i] = __ldcg(vg + i); pD[i] = __ldcg(vg + K + i); }
  // 4. C = R^{-1} X^T, own columns q (= own rows, C being symmetric)
  const int ncc = nrl;
  for (int idx = tid; idx < K * ncc; idx += nth) {
    const int i = idx / ncc, lq = idx - (idx / ncc) * ncc;
    const int q = rank + lq * SCL_NC;
    Xc[(size_t)i * ncc + lq] = q < K ? __ldcg(Xg + (size_t)q * K + i) : 0.0;
  }
  __syncthreads();
  scl_forward(K, ncc, Rp, rdiag, Xc);
  for (int idx = tid; idx < K * ncc; idx += nth) {
    const int i = idx / ncc, lq = idx - (idx / ncc) * ncc;
    Mr[(size_t)lq * K + i] = Xc[(size_t)i * ncc + lq];
  }
  __syncthreads();
  // 5. Householder tridiagonalisation on the distributed rows. Column k of
  //    the current matrix is its row k (symmetry): the owner of row k+1
  //    broadcasts that row with the partial products, and every CTA applies
  //    the step's rank-2 update to it, which gives column k+1 and the next
  //    reflector without a second exchange.
  double* uc = u;          // reflector of the current step
  double* un = fvec;       // reflector of the next step
  double* xn = colc;       // next column, below the diagonal
  double* wv = wk3;        // w of the current step
  __shared__ double s_hh[2];   // alpha of the current / next step (by parity)
  __shared__ double s_red[3];  // K, da, dd
  if (rank == 0)
    for (int j = tid; j < K - 1; j += nth)
      for (int r = 0; r < SCL_NC; ++r) cl.map_shared_rank(cbuf, r)[j] = Mr[1 + j];
  cl.sync();
  if (wid == 0) scl_reflector_warp(K - 1, cbuf, uc, &s_hh[0]);
  __syncthreads();
  for (int k = 0; k + 2 < K; ++k) {
    const int len = K - k - 1;
    const int par = k & 1;
    const bool more = k + 3 < K;
    double* pb = pbuf + (size_t)par * SCL_NC * K;
    double* rb = cbuf + (size_t)((k + 1) & 1) * K;
    const double alpha = s_hh[par];
    const int li0 = (k + 1 - rank > 0) ? (k + 1 - rank + SCL_NC - 1) / SCL_NC : 0;   // first own row > k
    // partial products over the own rows, sent to every CTA; row k+1 from its owner
    for (int j = tid; j < len; j += nth) {
      double acc = 0.0;
      for (int li = li0; li < nrl; ++li) {
        const int i = rank + li * SCL_NC;
        if (i >= K) break;
        acc += Mr[(size_t)li * K + k + 1 + j] * uc[i - k - 1];
      }
      for (int r = 0; r < SCL_NC; ++r) cl.map_shared_rank(pb, r)[(size_t)rank * K + j] = acc;
    }
    if (more && (k + 1) % SCL_NC == rank) {
      const double* row = Mr + (size_t)((k + 1) / SCL_NC) * K + k + 2;
      for (int j = tid; j < len - 1; j += nth)
        for (int r = 0; r < SCL_NC; ++r) cl.map_shared_rank(rb, r)[j] = row[j];
    }
    cl.sync();
    for (int j = tid; j < len; j += nth) {
      double t = 0.0;
      for (int r = 0; r < SCL_NC; ++r) t += pb[(size_t)r * K + j];
      p[j] = t;
    }
    __syncthreads();
    // K = u.p, da = u.p_A, dd = u.p_D, one warp each
    if (wid < 3) {
      const double* v = wid == 0 ? p : (wid == 1 ? pA + k + 1 : pD + k + 1);
      double acc = 0.0;
      for (int j = lane; j < len; j += 32) acc += uc[j] * v[j];
      acc = warp_sum(acc);
      if (lane == 0) s_red[wid] = acc;
    }
    __syncthreads();
    const double m2K = -2.0 * s_red[0], da = s_red[1], dd = s_red[2];
    // w = 2 p - 2 K u; the next column = row k+1 after this step's update
    const double u0 = uc[0], w0 = hh_w(m2K, u0, p[0]);
    for (int j = tid; j < len; j += nth) {
      const double wj = hh_w(m2K, uc[j], p[j]);
      wv[j] = wj;
      if (more && j >= 1) xn[j - 1] = hh_upd(rb[j - 1], u0, wj, w0, uc[j]);
    }
    __syncthreads();
    // the last warp forms the next reflector while the others update the rows
    const int nupd = more ? nwarp - 1 : nwarp;
    if (more && wid == nwarp - 1) {
      scl_reflector_warp(len - 1, xn, un, &s_hh[par ^ 1]);
    } else {
      for (int li = li0 + wid; li < nrl; li += nupd) {
        const int i = rank + li * SCL_NC;
        if (i >= K) break;
        const double ui = uc[i - k - 1], wi = wv[i - k - 1];
        double* Mi = Mr + (size_t)li * K + k + 1;
        for (int j = lane; j < len; j += 32) Mi[j] = hh_upd(Mi[j], ui, wv[j], wi, uc[j]);
      }
      for (int j = tid; j < len; j += nupd * 32) {
        pA[k + 1 + j] -= 2.0 * da * uc[j];
        pD[k + 1 + j] -= 2.0 * dd * uc[j];
      }
      if (tid == 0 && (k + 1) % SCL_NC == rank) Mr[(size_t)((k + 1) / SCL_NC) * K + k] = alpha;
    }
    __syncthreads();
    double* t = uc; uc = un; un = t;
  }
  // 6. T's diagonals from the row owners
  for (int li = tid; li < nrl; li += nth) {
    const int i = rank + li * SCL_NC;
    if (i >= K) continue;
    const double dv = Mr[(size_t)li * K + i];
    const double ev = i > 0 ? Mr[(size_t)li * K + i - 1] : 0.0;   // T[i][i-1] = eo[i-1]
    for (int r = 0; r < SCL_NC; ++r) {
      cl.map_shared_rank(dg, r)[i] = dv;
      if (i > 0) cl.map_shared_rank(eo, r)[i - 1] = ev;
    }
  }
  if (tid == 0) eo[K - 1] = 0.0;
  cl.sync();
  // From here every CTA holds T, p_A, p_D and runs the same control flow on
  // the same values; the symbol traces are split over the CTAs by pixel
  // range and the grid points by index, the pieces exchanged through
  // distributed shared memory (buffers alternate by parity so that one
  // exchange never overwrites the previous one while it is read).
  __shared__ double s_trx[2 * SEL_MAXPTS * SCL_NC];   // grid trace partials [parity][point][rank]
  __shared__ double s_num[2 * SEL_MAXPTS];            // grid numerators [parity][point]
  __shared__ double s_bx[2 * SCL_NC];                 // Brent trace partials [parity][rank]
  const int pix0 = (int)((size_t)a.npix * rank / SCL_NC);
  const int pix1 = (int)((size_t)a.npix * (rank + 1) / SCL_NC);
  // 7. w0 = T^{-1} p_A, f = p_A + p_D - w0, r0^2 (one Thomas sweep)
  if (tid == 0) {
    sel_tri_solve(K, dg, eo, pA, 0.0, p, u, 0.0);
    double pw = 0.0;
    for (int i = 0; i < K; ++i) {
      pw += pA[i] * u[i];
      fvec[i] = pA[i] + pD[i] - u[i];
    }
    s_bc[3] = pw;
  }
  __syncthreads();
  const double r02 = (a.bnorm2 - s_bc[3]) > 0.0 ? (a.bnorm2 - s_bc[3]) : 0.0;
  // 8. grid search with widening, then Brent (as k_gcv_select)
  const int npts = a.npts < SEL_MAXPTS ? a.npts : SEL_MAXPTS;
  double lo = a.lo, hi = a.hi;
  int ext = 0, jbest = 0;
  double fbest = 0.0, step = 0.0;
  for (;;) {
    const int gp = ext & 1;
    step = (hi - lo) / (npts - 1);
    for (int j = tid; j < npts; j += nth) s_gam[j] = pow(10.0, (j == npts - 1) ? hi : lo + j * step);
    __syncthreads();
    const bool tab = (ext == 0 && a.trace_tab);
    if (!tab) {
      sel_traces(a, nullptr, npts, s_gam, s_tr, sh, pix0, pix1);
      for (int idx = tid; idx < npts * SCL_NC; idx += nth) {
        const int j = idx / SCL_NC, r = idx - j * SCL_NC;
        cl.map_shared_rank(s_trx, r)[((size_t)gp * SEL_MAXPTS + j) * SCL_NC + rank] = s_tr[j];
      }
    }
    // this CTA's grid points j = rank, rank + SCL_NC, ..., one warp each
    for (int j = rank + wid * SCL_NC; j < npts; j += nwarp * SCL_NC) {
      double* sc4 = scratch + (size_t)j * 4 * K;
      const double num = sel_numerator_warp(K, dg, eo, fvec, r02, s_gam[j], sc4);
      if (lane < SCL_NC) cl.map_shared_rank(s_num, lane)[gp * SEL_MAXPTS + j] = num;
    }
    cl.sync();
    for (int j = tid; j < npts; j += nth) {
      double tr;
      if (tab) {
        tr = a.trace_tab[j];
      } else {
        tr = 0.0;
        for (int r = 0; r < SCL_NC; ++r) tr += s_trx[((size_t)gp * SEL_MAXPTS + j) * SCL_NC + r];
      }
      const double den = a.n - tr;
      s_f[j] = s_num[gp * SEL_MAXPTS + j] / (den * den);
    }
    __syncthreads();
    jbest = 0;
    fbest = s_f[0];
    for (int j = 1; j < npts; ++j)
      if (s_f[j] < fbest) { fbest = s_f[j]; jbest = j; }
    __syncthreads();
    if (jbest == 0 && ext < a.max_ext) { lo -= 4.0; ++ext; continue; }
    if (jbest == npts - 1 && ext < a.max_ext) { hi += 4.0; ++ext; continue; }
    break;
  }
  auto tgrid = [&](int j) { return (j == npts - 1) ? hi : lo + j * step; };
  int nev = 0;
  auto feval = [&](double t) -> double {
    const double gam = pow(10.0, t);
    const double num = sel_eval_tw(a, K, dg, eo, fvec, r02, gam, u, wk3, sh, &s_bc[2], pix0, pix1);
    const int bp = nev & 1;
    ++nev;
    if (tid < SCL_NC) cl.map_shared_rank(s_bx, tid)[bp * SCL_NC + rank] = s_bc[2];
    cl.sync();
    double tr = 0.0;
    for (int r = 0; r < SCL_NC; ++r) tr += s_bx[bp * SCL_NC + r];
    const double den = a.n - tr;
    return num / (den * den);
  };
  double A = tgrid(jbest > 0 ? jbest - 1 : 0);
  double B = tgrid(jbest < npts - 1 ? jbest + 1 : npts - 1);
  const double cgold = 0.5 * (3.0 - sqrt(5.0));
  const double sqeps = sqrt(2.220446049250313e-16);
  double x = A + cgold * (B - A), w = x, v = x;
  double fx = feval(x), fw = fx, fv = fx;
  double d = 0.0, e = 0.0;
  for (int nfev = 1; nfev < 500; ++nfev) {
    const double xm = 0.5 * (A + B);
    const double tol1 = sqeps * fabs(x) + a.tolx / 3.0;
    const double tol2 = 2.0 * tol1;
    if (fabs(x - xm) <= tol2 - 0.5 * (B - A)) break;
    bool golden = true;
    if (fabs(e) > tol1) {
      double r = (x - w) * (fx - fv);
      double q = (x - v) * (fx - fw);
      double pp = (x - v) * q - (x - w) * r;
      q = 2.0 * (q - r);
      if (q > 0.0) pp = -pp;
      q = fabs(q);
      const double etemp = e;
      e = d;
      if (fabs(pp) < fabs(0.5 * q * etemp) && pp > q * (A - x) && pp < q * (B - x)) {
        d = pp / q;
        const double uu = x + d;
        if ((uu - A) < tol2 || (B - uu) < tol2) d = (xm >= x) ? tol1 : -tol1;
        golden = false;
      }
    }
    if (golden) { e = (x < xm) ? (B - x) : (A - x); d = cgold * e; }
    const double uu = (fabs(d) >= tol1) ? x + d : x + (d > 0 ? tol1 : -tol1);
    const double fu = feval(uu);
    if (fu <= fx) {
      if (uu < x) B = x; else A = x;
      v = w; fv = fw; w = x; fw = fx; x = uu; fx = fu;
    } else {
      if (uu < x) A = uu; else B = uu;
      if (fu <= fw || w == x) { v = w; fv = fw; w = uu; fw = fu; }
      else if (fu <= fv || v == x || v == w) { v = uu; fv = fu; }
    }
  }
  const double tbest = (fx <= fbest) ? x : tgrid(jbest);
  if (tid == 0 && rank == 0) {
    a.out[0] = pow(10.0, tbest);
    a.out[1] = (double)ext;
    a.out[2] = (fx <= fbest) ? fx : fbest;
  }
}


// Up to three selections (k_gcv_select_cl args a0..a2) on gridDim.x /
// SCL_NC clusters: cluster c runs, in index order, the selections whose bits
// are set in bits [4c, 4c + 4) of `plan`. One cluster per selection gives
// the lowest latency; two small selections back to back on one cluster take
// about as long as one large one and leave the SMs to other work (the
// batched solver runs several GCVs at once). The results do not depend on
// the plan.
__global__ void __launch_bounds__(SCL_THREADS) k_gcv_select_cl(GcvSelectArgs a0, GcvSelectArgs a1, GcvSelectArgs a2,
                                                             unsigned plan) {
  namespace cg = cooperative_groups;
  cg::cluster_group cl = cg::this_cluster();
  const unsigned mask = (plan >> (4 * (blockIdx.x / SCL_NC))) & 15u;
  bool first = true;
  for (int q = 0; q < 3; ++q) {
    if (!(mask & (1u << q))) continue;
    if (!first) cl.sync();   // every CTA is done with the previous selection's shared memory
    sel_cl_run(q == 0 ? a0 : (q == 1 ? a1 : a2));
    first = false;
  }
}
}  // namespace db
