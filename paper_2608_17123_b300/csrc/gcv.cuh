// GCV choice of the regularisation parameter (Sec. 3, Eq. (xgamma), Eq. (GCV)).
//
// GCV(gamma) = ||A x_gamma - b||^2 / (n - tr(A A_gamma^{-1} A^T))^2.
// Projected form (this library's choice; the paper's dense GSVD does not
// scale past m ~ 64):
//  * numerator: x_gamma restricted to span(V), V = orthonormal basis of
//    K_k(A^T A, A^T b) (Lanczos on A^T A with two classical Gram-Schmidt
//    passes per step) plus orth(D^T c) when the shift c is non-zero.
//    G_A = V^T A^T A V, G_D = V^T D^T D V, g_A = V^T A^T b, g_D = V^T D^T c
//    are accumulated as the basis grows (double). The pair is reduced to
//    diagonal form Y^T G_A Y = diag(lam), Y^T (G_A + G_D) Y = I in double
//    (Cholesky, congruence, Householder tridiagonalisation, implicit QR),
//    after which the numerator is the sum of squares
//      sum_j [gamma (sqrt(lam_j) d_j - ahat_j (1-lam_j)) / (lam_j + gamma(1-lam_j))]^2 + r0^2.
//  * trace: the same pair under periodic boundary conditions,
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

// mean of w^2 over the valid gradient entries: sum via k_dot, divided on the host.

// ---- the small problem and the selection (one block) --------------------------
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
  const float* rho;       // [npix] symbol ratios
  int npix;
  double lo, hi, tolx;
  int npts, max_ext;
  double* work;           // >= 3 kk*kk + 8 kk doubles
  double* out;            // out[0] = gamma, out[1] = extensions, out[2] = GCV value
};

constexpr int SEL_THREADS = 1024;

__device__ double sel_block_sum(double v, double* sh) {
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  double s = (threadIdx.x < 32) ? sh[threadIdx.x] : 0.0;
  if (threadIdx.x < 32) s = warp_sum(s);
  __syncthreads();
  if (threadIdx.x == 0) sh[0] = s;
  __syncthreads();
  double r = sh[0];
  __syncthreads();
  return r;
}

// GCV at t = log10(gamma); all threads participate; returns the value in all.
__device__ double sel_eval(const GcvSelectArgs& a, double t, const double* lam, const double* sl,
                           const double* dd, const double* ahat, double r02, double* sh) {
  const double gamma = pow(10.0, t);
  // numerator: sum over the kk eigen-components
  double e2 = 0.0;
  for (int j = threadIdx.x; j < a.kk; j += blockDim.x) {
    const double den = lam[j] + gamma * (1.0 - lam[j]);
    const double e = gamma * (sl[j] * dd[j] - ahat[j] * (1.0 - lam[j])) / den;
    e2 += e * e;
  }
  // trace: float terms, Kahan-compensated per thread, double across threads
  const float gs = (float)(gamma * a.s);
  float sum = 0.f, comp = 0.f;
  for (int i = threadIdx.x; i < a.npix; i += blockDim.x) {
    const float term = __frcp_rn(1.0f + gs * a.rho[i]);
    const float y = term - comp;
    const float tt = sum + y;
    comp = (tt - sum) - y;
    sum = tt;
  }
  double part[1];
  const double num = sel_block_sum(e2, sh) + r02;
  const double tr = sel_block_sum((double)sum - (double)comp, sh);
  (void)part;
  const double den = a.n - tr;
  return num / (den * den);
}

__global__ void __launch_bounds__(SEL_THREADS) k_gcv_select(GcvSelectArgs a) {
  __shared__ double sh[64];
  __shared__ double s_val[4];
  const int kk = a.kk, ld = a.ld, tid = threadIdx.x, nth = blockDim.x;
  double* M = a.work;                 // kk x kk (row-major M[i*kk + j])
  double* C = M + kk * kk;            // kk x kk
  double* X = C + kk * kk;            // kk x kk
  double* pA = X + kk * kk;
  double* pD = pA + kk;
  double* lam = pD + kk;
  double* sl = lam + kk;
  double* ahat = sl + kk;
  double* dvec = ahat + kk;
  double* ev = dvec + kk;             // tridiagonal diag
  double* eo = ev + kk;               // tridiagonal off-diagonal
  auto GAe = [&](int i, int j) { return i <= j ? a.GA[(size_t)i * ld + j] : a.GA[(size_t)j * ld + i]; };
  auto GDe = [&](int i, int j) { return i <= j ? a.GD[(size_t)i * ld + j] : a.GD[(size_t)j * ld + i]; };
  // 1. M = G_A + G_D, C = G_A (full symmetric)
  for (int idx = tid; idx < kk * kk; idx += nth) {
    int i = idx / kk, j = idx % kk;
    M[idx] = GAe(i, j) + GDe(i, j);
    C[idx] = GAe(i, j);
  }
  __syncthreads();
  double maxdiag = 0.0;
  for (int i = 0; i < kk; ++i) maxdiag = fmax(maxdiag, M[i * kk + i]);
  // 2. Cholesky M = R R^T (lower, in place)
  for (int c = 0; c < kk; ++c) {
    if (tid == 0) {
      double piv = M[c * kk + c];
      double floor_ = 1e-14 * maxdiag;
      M[c * kk + c] = sqrt(piv > floor_ ? piv : floor_);
    }
    __syncthreads();
    const double rc = M[c * kk + c];
    for (int i = c + 1 + tid; i < kk; i += nth) M[i * kk + c] /= rc;
    __syncthreads();
    const int rem = kk - c - 1;
    for (int idx = tid; idx < rem * rem; idx += nth) {
      int i = c + 1 + idx / rem, j = c + 1 + idx % rem;
      if (j <= i) M[i * kk + j] -= M[i * kk + c] * M[j * kk + c];
    }
    __syncthreads();
  }
  // 3. X = R^{-1} G_A (column by column), pA = R^{-1} g_A, pD = R^{-1} g_D
  for (int q = tid; q < kk + 2; q += nth) {
    for (int i = 0; i < kk; ++i) {
      double s = q < kk ? C[i * kk + q] : (q == kk ? a.gA[i] : a.gD[i]);
      for (int l = 0; l < i; ++l) s -= M[i * kk + l] * (q < kk ? X[l * kk + q] : (q == kk ? pA[l] : pD[l]));
      s /= M[i * kk + i];
      if (q < kk) X[i * kk + q] = s; else if (q == kk) pA[i] = s; else pD[i] = s;
    }
  }
  __syncthreads();
  // 4. C = R^{-1} X^T  (= R^{-1} G_A R^{-T})
  for (int q = tid; q < kk; q += nth) {
    for (int i = 0; i < kk; ++i) {
      double s = X[q * kk + i];
      for (int l = 0; l < i; ++l) s -= M[i * kk + l] * C[l * kk + q];
      C[i * kk + q] = s / M[i * kk + i];
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
    const double nx = sqrt(nx2);
    if (nx2 - x0 * x0 <= 1e-300 * (1.0 + nx2)) {   // already tridiagonal in this column
      __syncthreads();
      continue;
    }
    const double alpha = x0 >= 0 ? -nx : nx;
    // u = x - alpha e1, normalised
    for (int i = tid; i < len; i += nth) u[i] = C[(k + 1 + i) * kk + k] - (i == 0 ? alpha : 0.0);
    __syncthreads();
    double pu = 0.0;
    for (int i = tid; i < len; i += nth) pu += u[i] * u[i];
    const double nu = sqrt(sel_block_sum(pu, sh));
    for (int i = tid; i < len; i += nth) u[i] /= nu;
    __syncthreads();
    // p = C22 u
    for (int i = tid; i < len; i += nth) {
      double s = 0.0;
      for (int j = 0; j < len; ++j) s += C[(k + 1 + i) * kk + (k + 1 + j)] * u[j];
      p[i] = s;
    }
    __syncthreads();
    double pk = 0.0;
    for (int i = tid; i < len; i += nth) pk += u[i] * p[i];
    const double K = sel_block_sum(pk, sh);
    // w = 2p - 2K u ; C22 -= u w^T + w u^T
    for (int idx = tid; idx < len * len; idx += nth) {
      int i = idx / len, j = idx % len;
      const double wi = 2.0 * p[i] - 2.0 * K * u[i], wj = 2.0 * p[j] - 2.0 * K * u[j];
      C[(k + 1 + i) * kk + (k + 1 + j)] -= u[i] * wj + wi * u[j];
    }
    // column / row k
    for (int i = tid; i < len; i += nth) {
      const double v = (i == 0) ? alpha : 0.0;
      C[(k + 1 + i) * kk + k] = v;
      C[k * kk + (k + 1 + i)] = v;
    }
    // reflect pA, pD
    double da = 0.0, dd = 0.0;
    for (int i = tid; i < len; i += nth) { da += u[i] * pA[k + 1 + i]; dd += u[i] * pD[k + 1 + i]; }
    da = sel_block_sum(da, sh);
    dd = sel_block_sum(dd, sh);
    for (int i = tid; i < len; i += nth) { pA[k + 1 + i] -= 2.0 * da * u[i]; pD[k + 1 + i] -= 2.0 * dd * u[i]; }
    __syncthreads();
  }
  for (int i = tid; i < kk; i += nth) {
    ev[i] = C[i * kk + i];
    eo[i] = (i + 1 < kk) ? C[(i + 1) * kk + i] : 0.0;
  }
  __syncthreads();
  // 6. implicit symmetric QR with Wilkinson shifts on (ev, eo); rotations applied to pA, pD.
  if (tid == 0) {
    int hi = kk - 1;
    int guard = 0;
    while (hi > 0 && guard < 60 * kk) {
      ++guard;
      // deflate
      if (fabs(eo[hi - 1]) <= 1e-15 * (fabs(ev[hi - 1]) + fabs(ev[hi]))) { eo[hi - 1] = 0.0; --hi; continue; }
      int lo = hi - 1;
      while (lo > 0 && fabs(eo[lo - 1]) > 1e-15 * (fabs(ev[lo - 1]) + fabs(ev[lo]))) --lo;
      // Wilkinson shift from the trailing 2x2
      const double dlt = 0.5 * (ev[hi - 1] - ev[hi]);
      const double b2 = eo[hi - 1] * eo[hi - 1];
      const double sgn = dlt >= 0 ? 1.0 : -1.0;
      const double mu = ev[hi] - b2 / (dlt + sgn * sqrt(dlt * dlt + b2));
      double xq = ev[lo] - mu, zq = eo[lo];
      for (int k = lo; k < hi; ++k) {
        // Givens rotation zeroing zq against xq
        double c, s;
        if (zq == 0.0) { c = 1.0; s = 0.0; }
        else if (fabs(zq) > fabs(xq)) { double tau = -xq / zq; s = 1.0 / sqrt(1.0 + tau * tau); c = s * tau; }
        else { double tau = -zq / xq; c = 1.0 / sqrt(1.0 + tau * tau); s = c * tau; }
        // T <- G^T T G on rows/cols k, k+1 (G = [c s; -s c])
        if (k > lo) eo[k - 1] = c * eo[k - 1] - s * zq;
        const double a11 = ev[k], a22 = ev[k + 1], a12 = eo[k];
        ev[k] = c * c * a11 - 2.0 * c * s * a12 + s * s * a22;
        ev[k + 1] = s * s * a11 + 2.0 * c * s * a12 + c * c * a22;
        eo[k] = c * s * (a11 - a22) + (c * c - s * s) * a12;
        if (k + 1 < hi) { xq = eo[k]; zq = -s * eo[k + 1]; eo[k + 1] = c * eo[k + 1]; }
        // accumulate: vectors in the eigenbasis, v <- G^T v
        const double ya = pA[k], za = pA[k + 1];
        pA[k] = c * ya - s * za; pA[k + 1] = s * ya + c * za;
        const double yd = pD[k], zd = pD[k + 1];
        pD[k] = c * yd - s * zd; pD[k + 1] = s * yd + c * zd;
      }
    }
  }
  __syncthreads();
  // 7. diagonal form
  for (int j = tid; j < kk; j += nth) {
    double l = ev[j];
    l = l < 0.0 ? 0.0 : (l > 1.0 ? 1.0 : l);
    lam[j] = l;
    sl[j] = sqrt(l);
    ahat[j] = l > 0.0 ? pA[j] / sqrt(l) : 0.0;
    dvec[j] = pD[j];
  }
  __syncthreads();
  double pr = 0.0;
  for (int j = tid; j < kk; j += nth) pr += ahat[j] * ahat[j];
  double r02 = a.bnorm2 - sel_block_sum(pr, sh);
  r02 = r02 > 0.0 ? r02 : 0.0;
  // 8. grid search (+ widening) and Brent refinement on t = log10(gamma)
  double lo = a.lo, hi = a.hi;
  int ext = 0, jbest = 0;
  double fbest = 0.0, step = 0.0;
  for (;;) {
    step = (hi - lo) / (a.npts - 1);
    jbest = 0;
    fbest = 0.0;
    for (int j = 0; j < a.npts; ++j) {
      const double t = (j == a.npts - 1) ? hi : lo + j * step;
      const double f = sel_eval(a, t, lam, sl, dvec, ahat, r02, sh);
      if (j == 0 || f < fbest) { fbest = f; jbest = j; }
    }
    if (jbest == 0 && ext < a.max_ext) { lo -= 4.0; ++ext; continue; }
    if (jbest == a.npts - 1 && ext < a.max_ext) { hi += 4.0; ++ext; continue; }
    break;
  }
  auto tgrid = [&](int j) { return (j == a.npts - 1) ? hi : lo + j * step; };
  double A = tgrid(jbest > 0 ? jbest - 1 : 0);
  double B = tgrid(jbest < a.npts - 1 ? jbest + 1 : a.npts - 1);
  // Brent (all threads run the same control flow; values are identical)
  const double cgold = 0.5 * (3.0 - sqrt(5.0));
  const double sqeps = sqrt(2.220446049250313e-16);
  double x = A + cgold * (B - A), w = x, v = x;
  double fx = sel_eval(a, x, lam, sl, dvec, ahat, r02, sh), fw = fx, fv = fx;
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
    const double fu = sel_eval(a, uu, lam, sl, dvec, ahat, r02, sh);
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
  (void)s_val;
}

}  // namespace db
