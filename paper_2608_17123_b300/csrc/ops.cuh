// Linear operators of the method on the device (sm_103a):
//  * blur A^(i) of every level as a sum of separable terms, each a pair of
//    per-row "circular band" matrices (exact for the zero-boundary fine blur
//    of Sec. 5 and for every Galerkin coarsening W^T A W of Sec. 4);
//  * gradient L and L^T (Sec. 4.2);
//  * low-pass restriction W^T, prolongation W and the blockwise Approach D
//    transfer (Sec. 4, Sec. 4.2);
//  * construction of the bands from a PSF (one-sided Jacobi SVD of the PSF,
//    so a rank-r PSF gives r separable terms) and their coarsening.
#pragma once
#include "common.cuh"

namespace db {

constexpr int TM = 32;        // tile rows (r, contiguous in memory)
constexpr int TN = 32;        // tile columns (c)
constexpr int TY = 8;         // blockDim.y; blockDim.x = 32
constexpr int PIX = TN / TY;  // output pixels per thread
constexpr int MAX_BAND = 96;  // widest band a tile kernel accepts

// Column (within the tile) of output pixel j of this thread: each thread owns
// PIX consecutive columns of row threadIdx.x, so the column pass can slide one
// register window over them.
__device__ __forceinline__ int pix_col(int j) { return PIX * (int)threadIdx.y + j; }

// One level operator: A = sum_t (Cc_t kron Cr_t), acting as X -> sum_t Cr_t X Cc_t^T.
// A 1-D factor C (m x m) is stored as B[r][k] = C[r, (r + dlo + k) mod m],
// k < w ("circular band"). The transposed band has dlo_T = -(dlo + w - 1) and
// B_T[r][k] = C[(r + dlo_T + k) mod m, r].
template <typename Acc>
struct BandOp {
  int m, nterms;
  int dlo, w;                 // same band shape for row and column factors
  const Acc* br;              // [t][m][w] row factors (act on r)
  const Acc* bc;              // [t][m][w] column factors (act on c)
  const Acc* brT;
  const Acc* bcT;
  // Level 0 of a PSF whose non-zero taps are fewer than the work of its
  // separable terms (a motion blur): the zero-boundary convolution applied
  // directly, (A X)(r, c) = sum_i w_i X(r - p_i, c - q_i), X = 0 outside.
  // ntaps = 0: the separable bands above.
  int ntaps = 0;
  const int* tap_pq = nullptr;   // (p + 128) << 8 | (q + 128)
  const Acc* tap_w = nullptr;
  // Level 0 of a separable PSF (FP32/BF16 LSQR): the same blur applied as a
  // direct Toeplitz convolution over a TMA-loaded, zero-filled window
  // (toep.cuh). tp: forward taps, row factors [t][w] then column factors
  // [t][w]. The bands above stay valid (and are used by the other kernels).
  int toep = 0;
  const Acc* tp = nullptr;
};

constexpr int MAX_TAPS = 961;   // taps of a 31 x 31 PSF

__host__ __device__ inline int band_pitch(int w) { return w | 1; }

// Tile geometry of one blur application (forward or transposed).
struct TileGeom {
  int dlo, w;   // effective band offsets
  int lo, hi;   // loaded halo relative offsets (lo <= min(dlo,-1), hi >= max(dlo+w-1, 1))
  int H;        // TM + hi - lo  (same for rows and columns since TM == TN)
};

template <typename Acc>
__host__ __device__ inline TileGeom tile_geom(const BandOp<Acc>& op, bool tr) {
  TileGeom g;
  g.w = op.w;
  g.dlo = tr ? -(op.dlo + op.w - 1) : op.dlo;
  g.lo = g.dlo < -1 ? g.dlo : -1;
  int top = g.dlo + g.w - 1;
  g.hi = top > 1 ? top : 1;
  g.H = TM + g.hi - g.lo;
  return g;
}

// Shared memory (in Acc elements) of the tile blur: x tile H*H, z H*TM,
// bands 2*TM*pitch.
__host__ __device__ inline int tile_smem_elems(int H, int w) {
  return H * H + H * TM + 2 * TM * band_pitch(w);
}

// Global -> register load; CG bypasses L1 (data written earlier in the same
// launch by other blocks).
template <bool CG, typename T>
__device__ __forceinline__ typename Traits<T>::Acc gload(const T* p) {
  if constexpr (CG) {
    if constexpr (sizeof(T) == 2) {
      unsigned short u = __ldcg(reinterpret_cast<const unsigned short*>(p));
      return to_acc(*reinterpret_cast<const T*>(&u));
    } else {
      return __ldcg(p);
    }
  } else {
    return to_acc(*p);
  }
}

constexpr int GATHER_BATCH = 12;   // loads a thread keeps in flight per gather batch

// Load X over the tile [r0+lo, r0+TM-1+hi] x [c0+lo, c0+TN-1+hi] (indices
// wrapped mod m) scaled by `scale`, into sx[col][row] (pitch H). Each thread
// issues a batch of GATHER_BATCH loads before its first shared-memory store,
// so the window costs one memory round trip per batch (one batch for bands
// up to 23 wide) rather than one per element.
template <bool CG, typename T, typename Acc>
__device__ __forceinline__ void gather_tile(const T* __restrict__ X, int m, int r0, int c0,
                                            const TileGeom& g, Acc scale, Acc* sx, bool zero_outside = false) {
  constexpr int NT = 32 * TY;
  const int tid = threadIdx.x + 32 * threadIdx.y;
  const int H = g.H, HH = H * H;
  const int dc = NT / H, dr = NT - dc * H;      // idx += NT  ->  (col, row) += (dc, dr), with carry
  int cc = tid / H, rr = tid - cc * H;
  const int rb = r0 + g.lo, cb = c0 + g.lo;
  for (int base = tid; base < HH; base += NT * GATHER_BATCH) {
    Acc v[GATHER_BATCH];
#pragma unroll
    for (int q = 0; q < GATHER_BATCH; ++q) {
      v[q] = Acc(0);
      const bool in = !zero_outside || ((unsigned)(rb + rr) < (unsigned)m && (unsigned)(cb + cc) < (unsigned)m);
      if (base + q * NT < HH && in) v[q] = gload<CG, T>(X + wrap(rb + rr, m) + (size_t)wrap(cb + cc, m) * m);
      rr += dr;
      cc += dc;
      if (rr >= H) { rr -= H; ++cc; }
    }
#pragma unroll
    for (int q = 0; q < GATHER_BATCH; ++q)
      if (base + q * NT < HH) sx[base + q * NT] = v[q] * scale;
  }
}

template <typename T, typename Acc>
__device__ __forceinline__ void load_tile(const T* __restrict__ X, int m, int r0, int c0,
                                          const TileGeom& g, Acc scale, Acc* sx, bool zero_outside = false) {
  gather_tile<false, T, Acc>(X, m, r0, c0, g, scale, sx, zero_outside);
}

// The direct taps of a sparse level-0 operator into shared memory (they take
// the place of the band rows): weights in sw, packed offsets in spq.
template <typename Acc>
__device__ __forceinline__ void load_taps(const BandOp<Acc>& op, Acc* sw, int* spq) {
  const int tid = threadIdx.x + 32 * threadIdx.y;
  for (int i = tid; i < op.ntaps; i += 32 * TY) {
    sw[i] = op.tap_w[i];
    spq[i] = op.tap_pq[i];
  }
}

// out[j] += (A x)(r, c) = sum_i w_i x(r - p_i, c - q_i) over the zero-filled
// window in sx, or (A^T x)(r, c) = sum_i w_i x(r + p_i, c + q_i); taps from
// load_taps (the caller synchronised after loading them).
template <typename Acc>
__device__ __forceinline__ void taps_conv(const BandOp<Acc>& op, bool tr, const TileGeom& g, const Acc* sx,
                                          const Acc* sw, const int* spq, Acc (&out)[PIX]) {
  const int H = g.H;
  const int lr = (int)threadIdx.x - g.lo;
  const int lc0 = pix_col(0) - g.lo;
  const int sgn = tr ? -1 : 1;
  for (int i = 0; i < op.ntaps; ++i) {
    const Acc wv = sw[i];
    const int pq = spq[i];
    const int dp = sgn * ((pq >> 8) - 128), dq = sgn * ((pq & 255) - 128);
    const Acc* base = sx + (lc0 - dq) * H + (lr - dp);
#pragma unroll
    for (int j = 0; j < PIX; ++j) out[j] += wv * base[j * H];
  }
}

// Bands of term t for the tile's rows / columns into shared memory (loads of
// a batch issued before the stores, as in gather_tile).
template <typename Acc>
__device__ __forceinline__ void load_bands(const BandOp<Acc>& op, bool tr, int t, int r0, int c0, const TileGeom& g,
                                           Acc* sbr, Acc* sbc) {
  constexpr int NT = 32 * TY, NB = 4;
  const int m = op.m, w = g.w, pw = band_pitch(w);
  const int tid = threadIdx.x + 32 * threadIdx.y;
  const Acc* BR = (tr ? op.brT : op.br) + (size_t)t * m * w;
  const Acc* BC = (tr ? op.bcT : op.bc) + (size_t)t * m * w;
  const int n = TM * w;
  for (int base = tid; base < n; base += NT * NB) {
    Acc a[NB], b[NB];
#pragma unroll
    for (int q = 0; q < NB; ++q) {
      const int idx = base + q * NT;
      a[q] = b[q] = Acc(0);
      if (idx < n) {
        const int rr = idx / w, k = idx - rr * w;
        a[q] = BR[(size_t)wrap(r0 + rr, m) * w + k];
        b[q] = BC[(size_t)wrap(c0 + rr, m) * w + k];
      }
    }
#pragma unroll
    for (int q = 0; q < NB; ++q) {
      const int idx = base + q * NT;
      if (idx < n) {
        const int rr = idx / w, k = idx - rr * w;
        sbr[rr * pw + k] = a[q];
        sbc[rr * pw + k] = b[q];
      }
    }
  }
}

// The two 1-D passes of one separable term. KW > 0: bands at most KW wide
// (KW = 16, or 32 in float working precision, where the taps fit the
// register budget), loops fully unrolled (every shared-memory load of an output issued before
// its FMAs, taps of step 1 held in registers, two partial sums); KW == 0:
// any width, runtime loop.
template <int KW, typename Acc>
__device__ __forceinline__ void conv_term(const TileGeom& g, const Acc* sx, Acc* sz, const Acc* sbr,
                                          const Acc* sbc, Acc (&out)[PIX]) {
  const int w = g.w, pw = band_pitch(w), H = g.H;
  const int r = threadIdx.x;
  // step 1: along r with the row factor, for every loaded column
  {
    const Acc* brow = sbr + r * pw;
    const int off = r - g.lo + g.dlo;
    if constexpr (KW > 0) {
      Acc bk[KW];
#pragma unroll
      for (int k = 0; k < KW; ++k) bk[k] = (k < w) ? brow[k] : Acc(0);
      for (int cz = threadIdx.y; cz < H; cz += TY) {
        const Acc* xs = sx + cz * H + off;
        Acc a0 = 0, a1 = 0;
#pragma unroll
        for (int k = 0; k < KW; k += 2) {
          if (k < w) a0 += bk[k] * xs[k];
          if (k + 1 < w) a1 += bk[k + 1] * xs[k + 1];
        }
        sz[cz * TM + r] = a0 + a1;
      }
    } else {
      for (int cz = threadIdx.y; cz < H; cz += TY) {
        const Acc* xs = sx + cz * H + off;
        Acc acc = 0;
#pragma unroll 4
        for (int k = 0; k < w; ++k) acc += brow[k] * xs[k];
        sz[cz * TM + r] = acc;
      }
    }
  }
  __syncthreads();
  // step 2: along c with the column factor, for this thread's PIX
  // consecutive columns (their windows share PIX + w - 1 rows of sz, read
  // once into registers in the unrolled form)
  const int cb = pix_col(0);
  if constexpr (KW > 0) {
    Acc zv[KW + PIX - 1];
    const Acc* zs0 = sz + (cb - g.lo + g.dlo) * TM + r;
#pragma unroll
    for (int q = 0; q < KW + PIX - 1; ++q) zv[q] = (q < w + PIX - 1) ? zs0[q * TM] : Acc(0);
#pragma unroll
    for (int j = 0; j < PIX; ++j) {
      const Acc* bcol = sbc + (cb + j) * pw;
      Acc a0 = 0, a1 = 0;
#pragma unroll
      for (int k = 0; k < KW; k += 2) {
        if (k < w) a0 += bcol[k] * zv[j + k];
        if (k + 1 < w) a1 += bcol[k + 1] * zv[j + k + 1];
      }
      out[j] += a0 + a1;
    }
  } else {
#pragma unroll
    for (int j = 0; j < PIX; ++j) {
      const int c = cb + j;
      const Acc* bcol = sbc + c * pw;
      const Acc* zs = sz + (c - g.lo + g.dlo) * TM + r;
      Acc acc = 0;
#pragma unroll 4
      for (int k = 0; k < w; ++k) acc += bcol[k] * zs[k * TM];
      out[j] += acc;
    }
  }
}

// out[j] += (A or A^T applied to the tile in sx) at pixel (r0+tx, c0+pix_col(j)).
// Caller has loaded sx (and synchronised). Uses sz/sb scratch.
// `first_loaded`: the caller already loaded term 0's bands (together with the
// tile, before one barrier).
template <typename Acc>
__device__ __forceinline__ void tile_conv(const BandOp<Acc>& op, bool tr, int r0, int c0,
                                          const TileGeom& g, const Acc* sx, Acc* sz, Acc* sbr,
                                          Acc* sbc, Acc (&out)[PIX], bool first_loaded = false) {
  if (op.ntaps > 0) {
    if (!first_loaded) {
      __syncthreads();
      load_taps<Acc>(op, sbr, reinterpret_cast<int*>(sbc));
    }
    __syncthreads();
    taps_conv<Acc>(op, tr, g, sx, sbr, reinterpret_cast<const int*>(sbc), out);
    return;
  }
  for (int t = 0; t < op.nterms; ++t) {
    if (!(t == 0 && first_loaded)) {
      __syncthreads();
      load_bands<Acc>(op, tr, t, r0, c0, g, sbr, sbc);
    }
    __syncthreads();
    if (g.w <= 16) conv_term<16, Acc>(g, sx, sz, sbr, sbc, out);
    else if (sizeof(Acc) == 4 && g.w <= 32) conv_term<sizeof(Acc) == 4 ? 32 : 0, Acc>(g, sx, sz, sbr, sbc, out);
    else conv_term<0, Acc>(g, sx, sz, sbr, sbc, out);
  }
}

// ---- standalone blur apply: Y = scale * A X (or A^T X) ----------------------
// `nrm2` (optional, device): the input is scaled by 1/sqrt(*nrm2) on load;
// `xcopy` (optional): the scaled input is also written there (own pixels).
template <typename T, typename Acc>
__global__ void __launch_bounds__(256) k_blur(BandOp<Acc> op, int tr, const T* __restrict__ X,
                                              T* __restrict__ Y, Acc scale, const double* nrm2 = nullptr,
                                              T* xcopy = nullptr) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Acc* sm = reinterpret_cast<Acc*>(smem_raw);
  const int m = op.m;
  const TileGeom g = tile_geom(op, tr != 0);
  Acc* sx = sm;
  Acc* sz = sx + g.H * g.H;
  Acc* sbr = sz + g.H * TM;
  Acc* sbc = sbr + TM * band_pitch(g.w);
  const int nt = (m + TM - 1) / TM;
  if (nrm2) scale = (Acc)(1.0 / sqrt(*nrm2));
  for (int tile = blockIdx.x; tile < nt * nt; tile += gridDim.x) {
    const int r0 = (tile % nt) * TM, c0 = (tile / nt) * TN;
    __syncthreads();
    load_tile<T, Acc>(X, m, r0, c0, g, scale, sx, op.ntaps > 0);
    Acc out[PIX] = {};
    tile_conv<Acc>(op, tr != 0, r0, c0, g, sx, sz, sbr, sbc, out);
    const int r = r0 + threadIdx.x;
#pragma unroll
    for (int j = 0; j < PIX; ++j) {
      const int c = c0 + pix_col(j);
      if (r < m && c < m) {
        Y[r + (size_t)c * m] = store_cast<T, Acc>(out[j]);
        if (xcopy) xcopy[r + (size_t)c * m] = store_cast<T, Acc>(sx[(pix_col(j) - g.lo) * g.H + threadIdx.x - g.lo]);
      }
    }
  }
}

// ---- gradient L, L^T, and D^T D = L^T diag(w^2) L -----------------------------
template <typename T>
__global__ void k_L(int m, const T* __restrict__ X, T* __restrict__ Qx, T* __restrict__ Qy) {
  using Acc = typename Traits<T>::Acc;
  size_t n = (size_t)m * m;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    int r = (int)(i % m), c = (int)(i / m);
    Acc xv = to_acc(X[i]);
    Acc qx = r < m - 1 ? to_acc(X[i + 1]) - xv : Acc(0);
    Acc qy = c < m - 1 ? to_acc(X[i + m]) - xv : Acc(0);
    Qx[i] = store_cast<T, Acc>(qx);
    Qy[i] = store_cast<T, Acc>(qy);
  }
}

template <typename T>
__global__ void k_Lt(int m, const T* __restrict__ Qx, const T* __restrict__ Qy, T* __restrict__ X) {
  using Acc = typename Traits<T>::Acc;
  size_t n = (size_t)m * m;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    int r = (int)(i % m), c = (int)(i / m);
    Acc s = 0;
    if (r < m - 1) s -= to_acc(Qx[i]);
    if (r > 0) s += to_acc(Qx[i - 1]);
    if (c < m - 1) s -= to_acc(Qy[i]);
    if (c > 0) s += to_acc(Qy[i - m]);
    X[i] = store_cast<T, Acc>(s);
  }
}

// Y = L^T diag(w^2) L X on Acc-typed vectors (w planes may be null = 1).
template <typename Acc, typename T>
__global__ void k_DtD(int m, const Acc* __restrict__ X, const T* __restrict__ Wx,
                      const T* __restrict__ Wy, Acc* __restrict__ Y) {
  size_t n = (size_t)m * m;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    int r = (int)(i % m), c = (int)(i / m);
    Acc xv = X[i];
    Acc s = 0;
    if (r < m - 1) { Acc q = X[i + 1] - xv; Acc ww = Wx ? to_acc(Wx[i]) : Acc(1); s -= ww * ww * q; }
    if (r > 0) { Acc q = xv - X[i - 1]; Acc ww = Wx ? to_acc(Wx[i - 1]) : Acc(1); s += ww * ww * q; }
    if (c < m - 1) { Acc q = X[i + m] - xv; Acc ww = Wy ? to_acc(Wy[i]) : Acc(1); s -= ww * ww * q; }
    if (c > 0) { Acc q = xv - X[i - m]; Acc ww = Wy ? to_acc(Wy[i - m]) : Acc(1); s += ww * ww * q; }
    Y[i] = s;
  }
}

// ---- wavelet transfers --------------------------------------------------------
struct Filter { int kappa; double h[4]; };

// Y (mc x mc) = W1^T X W1, W1^T[r, (2r+k) mod m] = h_k (Sec. 4).
template <typename T>
__global__ void k_restrict(int m, Filter f, const T* __restrict__ X, T* __restrict__ Y) {
  using Acc = typename Traits<T>::Acc;
  const int mc = m / 2;
  size_t nc = (size_t)mc * mc;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < nc; i += (size_t)gridDim.x * blockDim.x) {
    int r = (int)(i % mc), c = (int)(i / mc);
    Acc s = 0;
    for (int b = 0; b < f.kappa; ++b) {
      int cc = wrap(2 * c + b, m);
      Acc t = 0;
      for (int a = 0; a < f.kappa; ++a) t += (Acc)f.h[a] * to_acc(X[wrap(2 * r + a, m) + (size_t)cc * m]);
      s += (Acc)f.h[b] * t;
    }
    Y[i] = store_cast<T, Acc>(s);
  }
}

// X (m x m) = W1 Y W1^T with m = 2 mc. Fine index r receives h_a from coarse
// r' where (2r' + a) mod m = r. When `zero_row`/`zero_col` is set, the last
// fine row / column is written as 0 (Approach D planes: W~1 drops that row).
template <typename T>
__global__ void k_prolong(int mc, Filter f, const T* __restrict__ Y, T* __restrict__ X,
                          int zero_row, int zero_col) {
  using Acc = typename Traits<T>::Acc;
  const int m = 2 * mc;
  size_t n = (size_t)m * m;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    int r = (int)(i % m), c = (int)(i / m);
    if ((zero_row && r == m - 1) || (zero_col && c == m - 1)) { X[i] = store_cast<T, Acc>(Acc(0)); continue; }
    Acc s = 0;
    for (int b = (c & 1); b < f.kappa; b += 2) {
      const int cc = wrap((c - b) >> 1, mc);   // (2 cc + b) mod m == c
      Acc t = 0;
      for (int a = (r & 1); a < f.kappa; a += 2) {
        int rr = wrap((r - a) >> 1, mc);
        t += (Acc)f.h[a] * to_acc(Y[rr + (size_t)cc * mc]);
      }
      s += (Acc)f.h[b] * t;
    }
    X[i] = store_cast<T, Acc>(s);
  }
}

// Approach D: the transfer W~1 Q W1^T of a padded x-plane equals W1 Q W1^T
// on rows < m_f - 1 (the padded coarse row is zero) with the last row
// dropped; symmetrically for the y-plane.

// ---- band construction ----------------------------------------------------------
// Level 0: a 1-D factor f (length S, centred) is the zero-boundary Toeplitz
// C[r, s] = f[(r - s) + R] for 0 <= s < m; in band form (dlo = -R, w = S)
// B[r][k] = C[r, r + d], d = k - R, i.e. f[R - d] when 0 <= r + d < m.
// Coarse band: C'[r', s'] = sum_{a,b} h_a h_b C[(2r'+a) mod m, (2s'+b) mod m]
// (Sec. 4: A^(i+1) = W^T A^(i) W, factor by factor). Works in double.
__global__ void k_coarsen_bands(int m, int dlo, int w, int nterms, Filter f,
                                const double* __restrict__ B, int dlo2, int w2, double* __restrict__ B2) {
  const int mc = m / 2;
  size_t total = (size_t)nterms * mc * w2;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    int k2 = (int)(i % w2);
    int r2 = (int)((i / w2) % mc);
    int t = (int)(i / ((size_t)w2 * mc));
    int s2 = wrap(r2 + dlo2 + k2, mc);
    double acc = 0.0;
    for (int a = 0; a < f.kappa; ++a) {
      int ri = wrap(2 * r2 + a, m);
      for (int b = 0; b < f.kappa; ++b) {
        int sj = wrap(2 * s2 + b, m);
        int kk = wrap(sj - ri - dlo, m);   // offset index within a period
        if (kk < w) acc += f.h[a] * f.h[b] * B[((size_t)t * m + ri) * w + kk];
      }
    }
    B2[i] = acc;
  }
}

// Transposed band: B_T[r][k] = C[(r + dloT + k) mod m, r], dloT = -(dlo + w - 1).
template <typename Acc>
__global__ void k_transpose_band(int m, int dlo, int w, int nterms, const double* __restrict__ B,
                                 Acc* __restrict__ Bout, Acc* __restrict__ BTout) {
  const int dloT = -(dlo + w - 1);
  size_t total = (size_t)nterms * m * w;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    int k = (int)(i % w);
    int r = (int)((i / w) % m);
    int t = (int)(i / ((size_t)w * m));
    int s = wrap(r + dloT + k, m);           // row of C
    int kk = wrap(r - s - dlo, m);           // C[s, r] = B[s][r - s - dlo]
    BTout[i] = kk < w ? (Acc)B[((size_t)t * m + s) * w + kk] : Acc(0);
    Bout[i] = (Acc)B[i];
  }
}

// Fine bands in double (for coarsening) from 1-D factors.
__global__ void k_fine_bands_d(int m, int S, int nterms, const double* __restrict__ f,
                               double* __restrict__ B) {
  const int R = S / 2, w = S;
  size_t total = (size_t)nterms * m * w;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    int k = (int)(i % w);
    int r = (int)((i / w) % m);
    int t = (int)(i / ((size_t)w * m));
    int d = -R + k;
    bool in = (r + d >= 0) && (r + d < m);
    B[i] = in ? f[t * S + (R - d)] : 0.0;
  }
}

// ---- PSF factorisation: one-sided Jacobi SVD (Hestenes) in double -------------
// P (S x S, column-major P[p + q*S], p = row offset index) = sum_t s_t u_t v_t^T.
// Output: nterms, row factors fr[t][p] = s_t u_t(p), column factors fc[t][q] = v_t(q),
// for singular values above rel_tol * s_1. One block of 256 threads; S <= 64.
// Columns are rotated in tournament order: each round pairs every column with
// another (S/2 disjoint pairs, one warp per pair, lanes over the S rows), so a
// sweep is S-1 parallel rounds instead of S(S-1)/2 serial rotations.
__global__ void __launch_bounds__(256) k_psf_svd(int S, const double* __restrict__ P, double rel_tol, int* nterms,
                                                 double* fr, double* fc, double* work) {
  // work: U (S*S) columns = P's columns rotated, V (S*S), norms (S)
  double* U = work;
  double* V = work + S * S;
  double* nrm = work + 2 * S * S;
  __shared__ int s_rot;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarp = blockDim.x >> 5;
  for (int i = tid; i < S * S; i += blockDim.x) {
    U[i] = P[i];                       // columns of P, indexed U[p + q*S]
    V[i] = ((i % S) == (i / S)) ? 1.0 : 0.0;
  }
  const int np = S + (S & 1);          // players (one dummy when S is odd)
  for (int sweep = 0; sweep < 60; ++sweep) {
    if (tid == 0) s_rot = 0;
    __syncthreads();
    for (int round = 0; round < np - 1; ++round) {
      for (int k = warp; k < np / 2; k += nwarp) {
        // round-robin schedule: player 0 fixed, the others rotate
        const int a0 = k, b0 = np - 1 - k;
        int i = a0 == 0 ? 0 : 1 + (a0 - 1 + round) % (np - 1);
        int j = 1 + (b0 - 1 + round) % (np - 1);
        if (i >= S || j >= S) continue;          // dummy player
        if (i > j) { const int t = i; i = j; j = t; }
        double a = 0, b = 0, g = 0;
        for (int p = lane; p < S; p += 32) {
          const double ui = U[p + i * S], uj = U[p + j * S];
          a += ui * ui; b += uj * uj; g += ui * uj;
        }
        a = warp_sum(a); b = warp_sum(b); g = warp_sum(g);
        if (fabs(g) > 1e-300 && fabs(g) > 1e-15 * sqrt(a * b)) {
          const double zeta = (b - a) / (2.0 * g);
          const double t = (zeta >= 0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
          const double c = 1.0 / sqrt(1.0 + t * t), sn = c * t;
          for (int p = lane; p < S; p += 32) {
            const double ui = U[p + i * S], uj = U[p + j * S];
            U[p + i * S] = c * ui - sn * uj;
            U[p + j * S] = sn * ui + c * uj;
            const double vi = V[p + i * S], vj = V[p + j * S];
            V[p + i * S] = c * vi - sn * vj;
            V[p + j * S] = sn * vi + c * vj;
          }
          if (lane == 0) s_rot = 1;
        }
      }
      __syncthreads();
    }
    if (s_rot == 0) break;
    __syncthreads();
  }
  // P V = U (orthogonal columns): P = sum_j U_j V_j^T. Sort by norm.
  for (int j = warp; j < S; j += nwarp) {
    double a = 0;
    for (int p = lane; p < S; p += 32) a += U[p + j * S] * U[p + j * S];
    a = warp_sum(a);
    if (lane == 0) nrm[j] = sqrt(a);
  }
  __syncthreads();
  if (tid == 0) {
    double smax = 0;
    for (int j = 0; j < S; ++j) smax = fmax(smax, nrm[j]);
    int cnt = 0;
    for (int pass = 0; pass < S; ++pass) {
      int best = -1;
      double bv = -1;
      for (int j = 0; j < S; ++j)
        if (nrm[j] > bv) { bv = nrm[j]; best = j; }
      if (best < 0 || bv <= rel_tol * smax || bv <= 0.0) break;
      for (int p = 0; p < S; ++p) {
        fr[cnt * S + p] = U[p + best * S];     // s_t u_t
        fc[cnt * S + p] = V[p + best * S];     // v_t
      }
      nrm[best] = -2.0;
      ++cnt;
    }
    *nterms = cnt;
  }
}

}  // namespace db
