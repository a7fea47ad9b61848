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
// are kept as double-float pairs (float hi + float lo, error-free TwoSum) and
// the block that finishes last adds the chunks in a fixed order.
__device__ __forceinline__ void df_add(float& hi, float& lo, float xh, float xl) {
  const float s = hi + xh;
  const float bp = s - hi;
  const float e = (hi - (s - bp)) + (xh - bp);
  lo = lo + xl + e;
  hi = s;
}

// Kahan-compensated warp dot over strided elements, returned as (hi, lo).
__device__ __forceinline__ float2 warp_df(float acc, float comp) {
  // combine acc (with Kahan residue -comp) across the warp
  float hi = acc, lo = -comp;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float h2 = __shfl_xor_sync(0xffffffffu, hi, o);
    const float l2 = __shfl_xor_sync(0xffffffffu, lo, o);
    df_add(hi, lo, h2, l2);
  }
  return make_float2(hi, lo);
}

constexpr int VCH_E = 8;                 // elements per thread per chunk
constexpr int VCH_THREADS = 256;
constexpr int VCH_CHUNK = VCH_E * VCH_THREADS;
enum VchunkMode { VCH_UPDATE = 1, VCH_DOTS = 2, VCH_NORM = 4 };

// x -= sum_{i<nrows} coef[i*cstride] V_i (VCH_UPDATE); then V_i . x for
// i < nrows into out[i*ostride] (VCH_DOTS) and/or x . x into *outnorm
// (VCH_NORM). Float vectors only (the Krylov basis is held in working
// precision); part needs (nrows + 1) * gridDim.x float2.
__global__ void __launch_bounds__(VCH_THREADS) k_vchunk(size_t n, int nrows, const float* __restrict__ V, size_t ldv,
    const double* __restrict__ coef, int cstride, float* __restrict__ x, int mode, float2* __restrict__ part,
    unsigned* cnt, double* out, int ostride, double* outnorm, int E) {
  __shared__ float xs[VCH_CHUNK];
  __shared__ float cs[512];
  __shared__ int s_last;
  const int nch = gridDim.x, ch = blockIdx.x;
  const int CH = E * VCH_THREADS;
  const size_t beg = (size_t)ch * CH;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = VCH_THREADS / 32;
  if (mode & VCH_UPDATE)
    for (int i = tid; i < nrows; i += VCH_THREADS) cs[i] = (float)coef[(size_t)i * cstride];
  __syncthreads();
  float nacc = 0.f, ncomp = 0.f;
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
      const float y = xv * xv - ncomp;
      const float t = nacc + y;
      ncomp = (t - nacc) - y;
      nacc = t;
    }
    xs[le] = xv;
  }
  __syncthreads();
  if (mode & VCH_DOTS) {
    for (int i = wid; i < nrows; i += nw) {
      const float* vi = V + (size_t)i * ldv + beg;
      float acc = 0.f, comp = 0.f;
      for (int le = lane; le < CH; le += 32) {
        if (beg + le >= n) break;
        const float y = vi[le] * xs[le] - comp;
        const float t = acc + y;
        comp = (t - acc) - y;
        acc = t;
      }
      const float2 r = warp_df(acc, comp);
      if (lane == 0) part[(size_t)i * nch + ch] = r;
    }
  }
  if (mode & VCH_NORM) {
    const float2 r = warp_df(nacc, ncomp);
    __shared__ float2 wn[8];
    if (lane == 0) wn[wid] = r;
    __syncthreads();
    if (tid == 0) {
      float hi = 0.f, lo = 0.f;
      for (int w = 0; w < nw; ++w) df_add(hi, lo, wn[w].x, wn[w].y);
      part[(size_t)nrows * nch + ch] = make_float2(hi, lo);
    }
  }
  __syncthreads();
  if (tid == 0) {
    __threadfence();
    s_last = (atomicAdd(cnt, 1u) == (unsigned)nch - 1);
    __threadfence();
  }
  __syncthreads();
  if (!s_last) return;
  const int r0 = (mode & VCH_DOTS) ? 0 : nrows;
  const int r1 = (mode & VCH_NORM) ? nrows + 1 : nrows;
  for (int r = r0 + tid; r < r1; r += VCH_THREADS) {
    float hi = 0.f, lo = 0.f;
    for (int c = 0; c < nch; ++c) {
      const float2 pv = __ldcg(&part[(size_t)r * nch + c]);
      df_add(hi, lo, pv.x, pv.y);
    }
    const double v = (double)hi + (double)lo;
    if (r < nrows) out[(size_t)r * ostride] = v; else *outnorm = v;
  }
  if (tid == 0) *cnt = 0;
}

// Gram column j: with y = L^T diag(w^2) L v_j (computed here),
//   GA[i*ld + j] = V_i . t, GD[i*ld + j] = V_i . y (i <= j),
//   gA[j] = atb . v_j, gD[j] = dtc . v_j (dtc may be null -> 0).
template <typename T>
__global__ void __launch_bounds__(VCH_THREADS) k_gram_col(int m, int j, const float* __restrict__ V,
    const float* __restrict__ t, const T* __restrict__ wx, const T* __restrict__ wy, const float* __restrict__ atb,
    const float* __restrict__ dtc, float2* __restrict__ part, unsigned* cnt, double* GA, double* GD, int ld,
    double* gA, double* gD, int E) {
  __shared__ float ts[VCH_CHUNK];
  __shared__ float ys[VCH_CHUNK];
  __shared__ int s_last;
  const size_t n = (size_t)m * m;
  const int nch = gridDim.x, ch = blockIdx.x;
  const int CH = E * VCH_THREADS;
  const size_t beg = (size_t)ch * CH;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = VCH_THREADS / 32;
  const float* vj = V + (size_t)j * n;
  for (int k = 0; k < E; ++k) {
    const int le = k * VCH_THREADS + tid;
    const size_t i = beg + le;
    float tv = 0.f, yv = 0.f;
    if (i < n) {
      tv = t[i];
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
  const int nrows = j + 1;
  // rows 0..j: two dots each (slots 2i, 2i+1); row j+1: atb.v_j and dtc.v_j
  for (int i = wid; i <= nrows; i += nw) {
    float a1 = 0.f, c1 = 0.f, a2 = 0.f, c2 = 0.f;
    for (int le = lane; le < CH; le += 32) {
      if (beg + le >= n) break;
      float p1, q1, p2, q2;
      if (i < nrows) { const float vv = V[(size_t)i * n + beg + le]; p1 = vv; q1 = ts[le]; p2 = vv; q2 = ys[le]; }
      else { const float vv = vj[beg + le]; p1 = atb[beg + le]; q1 = vv; p2 = dtc ? dtc[beg + le] : 0.f; q2 = vv; }
      float y = p1 * q1 - c1, tt = a1 + y; c1 = (tt - a1) - y; a1 = tt;
      y = p2 * q2 - c2; tt = a2 + y; c2 = (tt - a2) - y; a2 = tt;
    }
    const float2 r1 = warp_df(a1, c1), r2 = warp_df(a2, c2);
    if (lane == 0) {
      part[(size_t)(2 * i) * nch + ch] = r1;
      part[(size_t)(2 * i + 1) * nch + ch] = r2;
    }
  }
  __syncthreads();
  if (tid == 0) {
    __threadfence();
    s_last = (atomicAdd(cnt, 1u) == (unsigned)nch - 1);
    __threadfence();
  }
  __syncthreads();
  if (!s_last) return;
  for (int sidx = tid; sidx < 2 * (nrows + 1); sidx += VCH_THREADS) {
    float hi = 0.f, lo = 0.f;
    for (int c = 0; c < nch; ++c) {
      const float2 pv = __ldcg(&part[(size_t)sidx * nch + c]);
      df_add(hi, lo, pv.x, pv.y);
    }
    const double v = (double)hi + (double)lo;
    const int i = sidx >> 1;
    if (i < nrows) {
      if ((sidx & 1) == 0) GA[(size_t)i * ld + j] = v; else GD[(size_t)i * ld + j] = v;
    } else {
      if ((sidx & 1) == 0) gA[j] = v; else gD[j] = v;
    }
  }
  if (tid == 0) *cnt = 0;
}

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
// tridiagonal SPD system, one Thomas sweep per gamma); the residual is
// evaluated without cancellation as gamma^2 u^T T u + r0^2 (sel_numerator).
// The trace is either the symbol trace (projected mode) or, when the basis is
// the whole space (exact mode, tiny levels), sum_j lam_j / (lam_j + gamma (1 - lam_j))
// over the eigenvalues of T (bisection with Sturm counts).
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
  double* work;           // >= 3 kk*kk + (6 + 2*SEL_MAXPTS + 1) kk doubles
  double* out;            // out[0] = gamma, out[1] = extensions, out[2] = GCV value
};

constexpr int SEL_THREADS = 512;

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
constexpr int SEL_MAXPTS = 64;

__device__ double sel_block_sum(double v, double* sh) {
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  double s = (threadIdx.x < 32 && threadIdx.x < (blockDim.x >> 5)) ? sh[threadIdx.x] : 0.0;
  if (threadIdx.x < 32) s = warp_sum(s);
  __syncthreads();
  if (threadIdx.x == 0) sh[0] = s;
  __syncthreads();
  double r = sh[0];
  __syncthreads();
  return r;
}

// Solve ((1 - gamma) T + gamma I) u = f by one Thomas sweep (T symmetric
// tridiagonal: diagonal d, off-diagonal e; the matrix is SPD for gamma > 0
// and for gamma = 0 when T is). cw is scratch of length kk.
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

// Trace term for a set of gammas (all threads); returns per-gamma traces in tr[].
__device__ void sel_traces(const GcvSelectArgs& a, const double* lam, int ng, const double* gam, double* tr,
                           double* sh) {
  for (int g = 0; g < ng; ++g) {
    double part = 0.0;
    if (a.exact) {
      for (int j = threadIdx.x; j < a.kk; j += blockDim.x) {
        const double l = lam[j];
        part += l / (l + gam[g] * (1.0 - l));
      }
    } else {
      const float gs = (float)(gam[g] * a.s);
      float sum = 0.f, comp = 0.f;
      for (int i = threadIdx.x; i < a.npix; i += blockDim.x) {
        const float term = __frcp_rn(1.0f + gs * a.rho[i]);
        const float y = term - comp;
        const float t = sum + y;
        comp = (t - sum) - y;
        sum = t;
      }
      part = (double)sum - (double)comp;
    }
    tr[g] = sel_block_sum(part, sh);
  }
}

__global__ void __launch_bounds__(SEL_THREADS) k_gcv_select(GcvSelectArgs a) {
  __shared__ double sh[64];
  __shared__ double s_gam[SEL_MAXPTS], s_tr[SEL_MAXPTS], s_f[SEL_MAXPTS];
  const int kk = a.kk, ld = a.ld, tid = threadIdx.x, nth = blockDim.x;
  double* M = a.work;                 // kk x kk (row-major M[i*kk + j])
  double* C = M + kk * kk;            // kk x kk
  double* X = C + kk * kk;            // kk x kk
  double* pA = X + kk * kk;
  double* pD = pA + kk;
  double* dg = pD + kk;               // tridiagonal diagonal
  double* eo = dg + kk;               // tridiagonal off-diagonal
  double* lam = eo + kk;              // eigenvalues of T (exact mode)
  double* scratch = lam + 2 * kk;     // per-thread Thomas scratch for the grid: SEL_MAXPTS * 2 kk
  auto GAe = [&](int i, int j) { return i <= j ? a.GA[(size_t)i * ld + j] : a.GA[(size_t)j * ld + i]; };
  auto GDe = [&](int i, int j) { return i <= j ? a.GD[(size_t)i * ld + j] : a.GD[(size_t)j * ld + i]; };
  // 1. M = G_A + G_D, C = G_A (full symmetric)
  for (int idx = tid; idx < kk * kk; idx += nth) {
    int i = idx / kk, j = idx % kk;
    M[idx] = GAe(i, j) + GDe(i, j);
    C[idx] = GAe(i, j);
  }
  __syncthreads();
  __shared__ double s_md;
  if (tid == 0) {
    double md = 0.0;
    for (int i = 0; i < kk; ++i) md = fmax(md, M[i * kk + i]);
    s_md = md;
  }
  __syncthreads();
  const double md = s_md;
  const double piv_floor = 1e-14 * md;
  // 2. Cholesky M = R R^T (lower, in place); rdiag = 1 / diag(R)
  double* rdiag = lam + kk;           // kk entries before the Thomas scratch
  __shared__ double s_rc;
  for (int c = 0; c < kk; ++c) {
    if (tid == 0) {
      const double piv = M[c * kk + c];
      const double r = sqrt(piv > piv_floor ? piv : piv_floor);
      M[c * kk + c] = r;
      s_rc = 1.0 / r;
      rdiag[c] = s_rc;
    }
    __syncthreads();
    const double rc = s_rc;
    for (int i = c + 1 + tid; i < kk; i += nth) M[i * kk + c] *= rc;
    __syncthreads();
    const int rem = kk - c - 1;
    for (int idx = tid; idx < rem * rem; idx += nth) {
      const int i = c + 1 + idx / rem, j = c + 1 + idx % rem;
      if (j <= i) M[i * kk + j] -= M[i * kk + c] * M[j * kk + c];
    }
    __syncthreads();
  }
  // 3. X = R^{-1} G_A, pA = R^{-1} g_A, pD = R^{-1} g_D (one column per thread,
  //    four partial sums to shorten the dependent chain)
  for (int q = tid; q < kk + 2; q += nth) {
    for (int i = 0; i < kk; ++i) {
      double s0 = q < kk ? C[i * kk + q] : (q == kk ? a.gA[i] : a.gD[i]);
      double s1 = 0.0, s2 = 0.0, s3 = 0.0;
      int l = 0;
      for (; l + 3 < i; l += 4) {
        const double x0 = q < kk ? X[l * kk + q] : (q == kk ? pA[l] : pD[l]);
        const double x1 = q < kk ? X[(l + 1) * kk + q] : (q == kk ? pA[l + 1] : pD[l + 1]);
        const double x2 = q < kk ? X[(l + 2) * kk + q] : (q == kk ? pA[l + 2] : pD[l + 2]);
        const double x3 = q < kk ? X[(l + 3) * kk + q] : (q == kk ? pA[l + 3] : pD[l + 3]);
        s0 -= M[i * kk + l] * x0; s1 -= M[i * kk + l + 1] * x1;
        s2 -= M[i * kk + l + 2] * x2; s3 -= M[i * kk + l + 3] * x3;
      }
      for (; l < i; ++l) s0 -= M[i * kk + l] * (q < kk ? X[l * kk + q] : (q == kk ? pA[l] : pD[l]));
      const double v = ((s0 + s1) + (s2 + s3)) * rdiag[i];
      if (q < kk) X[i * kk + q] = v; else if (q == kk) pA[i] = v; else pD[i] = v;
    }
  }
  __syncthreads();
  // 4. C = R^{-1} X^T  (= R^{-1} G_A R^{-T})
  for (int q = tid; q < kk; q += nth) {
    for (int i = 0; i < kk; ++i) {
      double s0 = X[q * kk + i], s1 = 0.0, s2 = 0.0, s3 = 0.0;
      int l = 0;
      for (; l + 3 < i; l += 4) {
        s0 -= M[i * kk + l] * C[l * kk + q]; s1 -= M[i * kk + l + 1] * C[(l + 1) * kk + q];
        s2 -= M[i * kk + l + 2] * C[(l + 2) * kk + q]; s3 -= M[i * kk + l + 3] * C[(l + 3) * kk + q];
      }
      for (; l < i; ++l) s0 -= M[i * kk + l] * C[l * kk + q];
      C[i * kk + q] = ((s0 + s1) + (s2 + s3)) * rdiag[i];
    }
  }
  __syncthreads();
  for (int idx = tid; idx < kk * kk; idx += nth) {   // symmetrise
    int i = idx / kk, j = idx % kk;
    if (i < j) { double v = 0.5 * (C[i * kk + j] + C[j * kk + i]); C[i * kk + j] = v; C[j * kk + i] = v; }
  }
  __syncthreads();
  // 5. Householder tridiagonalisation C = Q T Q^T; pA, pD <- Q^T pA, Q^T pD.
  double* u = X;            // reuse X rows as scratch vectors
  double* p = X + kk;
  for (int k = 0; k + 2 < kk; ++k) {
    const int len = kk - k - 1;
    double part = 0.0;
    for (int i = tid; i < len; i += nth) { double xv = C[(k + 1 + i) * kk + k]; part += xv * xv; }
    const double nx2 = sel_block_sum(part, sh);
    const double x0 = C[(k + 1) * kk + k];
    if (nx2 - x0 * x0 <= 1e-300 * (1.0 + nx2)) continue;   // column already reduced
    // u = (x - alpha e1) / ||x - alpha e1||, ||x - alpha e1||^2 = 2 nx (nx + |x0|)
    __shared__ double s_alpha, s_inu;
    if (tid == 0) {
      const double nx = sqrt(nx2);
      s_alpha = x0 >= 0 ? -nx : nx;
      s_inu = 1.0 / sqrt(2.0 * nx * (nx + fabs(x0)));
    }
    __syncthreads();
    const double alpha = s_alpha, inv_nu = s_inu;
    for (int i = tid; i < len; i += nth) u[i] = (C[(k + 1 + i) * kk + k] - (i == 0 ? alpha : 0.0)) * inv_nu;
    __syncthreads();
    for (int i = tid; i < len; i += nth) {
      const double* row = C + (size_t)(k + 1 + i) * kk + (k + 1);
      double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
      int j = 0;
      for (; j + 3 < len; j += 4) { s0 += row[j] * u[j]; s1 += row[j + 1] * u[j + 1]; s2 += row[j + 2] * u[j + 2]; s3 += row[j + 3] * u[j + 3]; }
      for (; j < len; ++j) s0 += row[j] * u[j];
      p[i] = (s0 + s1) + (s2 + s3);
    }
    __syncthreads();
    double pk = 0.0, da = 0.0, dd = 0.0;
    for (int i = tid; i < len; i += nth) { pk += u[i] * p[i]; da += u[i] * pA[k + 1 + i]; dd += u[i] * pD[k + 1 + i]; }
    const double K = sel_block_sum(pk, sh);
    da = sel_block_sum(da, sh);
    dd = sel_block_sum(dd, sh);
    for (int idx = tid; idx < len * len; idx += nth) {
      const int i = idx / len, j = idx % len;
      const double wi = 2.0 * p[i] - 2.0 * K * u[i], wj = 2.0 * p[j] - 2.0 * K * u[j];
      C[(k + 1 + i) * kk + (k + 1 + j)] -= u[i] * wj + wi * u[j];
    }
    for (int i = tid; i < len; i += nth) {
      const double v = (i == 0) ? alpha : 0.0;
      C[(k + 1 + i) * kk + k] = v;
      C[k * kk + (k + 1 + i)] = v;
      pA[k + 1 + i] -= 2.0 * da * u[i];
      pD[k + 1 + i] -= 2.0 * dd * u[i];
    }
    __syncthreads();
  }
  for (int i = tid; i < kk; i += nth) {
    dg[i] = C[i * kk + i];
    eo[i] = (i + 1 < kk) ? C[(i + 1) * kk + i] : 0.0;
  }
  __syncthreads();
  // 5b. w0 = T^{-1} p_A, f = p_A + p_D - w0, r0^2 = ||b||^2 - p_A . w0
  double* fvec = scratch + (size_t)SEL_MAXPTS * 2 * kk;     // kk
  __shared__ double s_r02;
  if (tid == 0) {
    double* w0 = scratch;
    sel_tri_solve(kk, dg, eo, pA, 0.0, scratch + kk, w0, 0.0);
    double pw = 0.0;
    for (int i = 0; i < kk; ++i) {
      pw += pA[i] * w0[i];
      fvec[i] = pA[i] + pD[i] - w0[i];
    }
    const double r = a.bnorm2 - pw;
    s_r02 = r > 0.0 ? r : 0.0;
  }
  __syncthreads();
  const double r02 = s_r02;
  // 6. exact mode: eigenvalues of T by bisection (Sturm counts), one per thread
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
  // 7. grid search (parallel over the grid points) with widening, then Brent
  const int npts = a.npts < SEL_MAXPTS ? a.npts : SEL_MAXPTS;
  double lo = a.lo, hi = a.hi;
  int ext = 0, jbest = 0;
  double fbest = 0.0, step = 0.0;
  for (;;) {
    step = (hi - lo) / (npts - 1);
    for (int j = tid; j < npts; j += nth) s_gam[j] = pow(10.0, (j == npts - 1) ? hi : lo + j * step);
    __syncthreads();
    sel_traces(a, lam, npts, s_gam, s_tr, sh);
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
  auto feval = [&](double t) -> double {
    __syncthreads();
    if (tid == 0) s_gam[0] = pow(10.0, t);
    __syncthreads();
    sel_traces(a, lam, 1, s_gam, s_tr, sh);
    if (tid == 0) {
      const double num = sel_numerator(kk, dg, eo, fvec, r02, s_gam[0], scratch, scratch + kk);
      const double den = a.n - s_tr[0];
      s_f[0] = num / (den * den);
    }
    __syncthreads();
    const double f = s_f[0];
    __syncthreads();
    return f;
  };
  double A = tgrid(jbest > 0 ? jbest - 1 : 0);
  double B = tgrid(jbest < npts - 1 ? jbest + 1 : npts - 1);
  // Brent (golden section + parabolic interpolation); every thread runs the
  // same control flow on the same broadcast values.
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

}  // namespace db
