// Level-0 blur of a separable PSF as a direct 2-D convolution (Sec. 5: the
// fine operator is the zero-boundary blur, A X = sum_t Cr_t X Cc_t^T with
// Toeplitz factors), used by the LSQR passes on FP32/BF16 storage.
//
// Every row of a Toeplitz factor's band holds the same taps, so the taps of
// both 1-D passes sit in registers and each pass slides a register window
// along its direction: one shared-memory load feeds w FMAs instead of one.
// The tile's halo window arrives by one TMA box copy whose out-of-bounds
// fill is the zero boundary (rows and columns outside [0, m) read 0), so no
// index is wrapped or clamped.
//
// Window of the tile (r0, c0): box rows r0 + f8 .. r0 + f8 + RB - 1 (f8 = dlo
// rounded down to a multiple of 8, so the box's innermost coordinate is
// 16-byte aligned for 2- and 4-byte elements; RB a multiple of 8) and box
// columns c0 + dlo .. c0 + dlo + CB - 1, CB = TN + w - 1, stored column by
// column with pitch RB. The forward and the transposed blur use the same
// window (the PSF side is odd, so the transposed band starts at dlo as well)
// with the taps reversed.
//
// Output mapping of the passes (256 threads): thread tid owns rows
// r0 + 4a .. r0 + 4a + 3 of column c0 + cl, a = tid % 8, cl = tid / 8, so its
// pointwise loads and stores are single 16-byte (FP32) or 8-byte (BF16)
// vector accesses.
#pragma once
#include "ops.cuh"
#include "tma.cuh"

namespace db {

constexpr int TOEP_MAX_W = 32;   // widest band of the direct path (taps in registers)

struct ToepGeom {
  int f8;   // first box row relative to r0 (a multiple of 8, <= dlo)
  int s;    // dlo - f8: box row of r0 + dlo
  int RB;   // box rows (multiple of 8)
  int CB;   // box columns
  int ZP;   // pitch of the intermediate (column pass output), 1 mod 32
};

__host__ __device__ inline ToepGeom toep_geom(int dlo, int w) {
  ToepGeom g;
  g.f8 = dlo >= 0 ? (dlo & ~7) : -((-dlo + 7) & ~7);
  g.s = dlo - g.f8;
  g.RB = (g.s + TM + w - 1 + 7) & ~7;
  g.CB = TN + w - 1;
  g.ZP = ((g.RB + 31) & ~31) + 1;
  return g;
}

// Shared memory of the direct path: alignment slack, the window (sized for
// 4-byte elements whatever the storage), the column-pass output and
// TOEP_SLOTS staging slots of the tile's pointwise operands (one vector each,
// column by column, 33 columns: c0 - 1 .. c0 + 31), then the taps.
constexpr int TOEP_SLOTS = 7;   // warps 0..6 fill one slot each, warp 7 the taps
static_assert(TOEP_SLOTS == TY - 1, "one staging warp per slot plus one for the taps");
constexpr int TOEP_SLOT_BYTES = (TN + 1) * TM * 4;
__host__ __device__ inline int toep_win_bytes(const ToepGeom& g) { return (g.RB * g.CB * 4 + 127) & ~127; }
__host__ __device__ inline int toep_z_bytes(const ToepGeom& g) { return (TN * g.ZP * 4 + 127) & ~127; }
// taps of every term (2 * nterms * w floats, nterms * w <= TOEP_MAX_TAPS)
constexpr int TOEP_MAX_TAPS = 1024;
constexpr int TOEP_TAP_BYTES = 2 * TOEP_MAX_TAPS * 4;
__host__ __device__ inline int toep_smem_bytes(const ToepGeom& g) {
  return 128 + toep_win_bytes(g) + toep_z_bytes(g) + TOEP_SLOTS * TOEP_SLOT_BYTES + TOEP_TAP_BYTES;
}

// ---- 4-element vector accesses (4 consecutive rows of one column) ----------
__device__ __forceinline__ void ld4cg(const float* p, float (&o)[4]) {
  const float4 v = __ldcg(reinterpret_cast<const float4*>(p));
  o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
}
__device__ __forceinline__ void ld4cg(const __nv_bfloat16* p, float (&o)[4]) {
  const uint2 v = __ldcg(reinterpret_cast<const uint2*>(p));
  o[0] = __uint_as_float(v.x << 16); o[1] = __uint_as_float(v.x & 0xffff0000u);
  o[2] = __uint_as_float(v.y << 16); o[3] = __uint_as_float(v.y & 0xffff0000u);
}
// read-only data of the launch (weights)
__device__ __forceinline__ void ld4nc(const float* p, float (&o)[4]) {
  const float4 v = __ldg(reinterpret_cast<const float4*>(p));
  o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
}
__device__ __forceinline__ void ld4nc(const __nv_bfloat16* p, float (&o)[4]) {
  const uint2 v = __ldg(reinterpret_cast<const uint2*>(p));
  o[0] = __uint_as_float(v.x << 16); o[1] = __uint_as_float(v.x & 0xffff0000u);
  o[2] = __uint_as_float(v.y << 16); o[3] = __uint_as_float(v.y & 0xffff0000u);
}
__device__ __forceinline__ void st4(float* p, const float (&v)[4]) {
  *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
}
__device__ __forceinline__ void st4(__nv_bfloat16* p, const float (&v)[4]) {
  const __nv_bfloat162 lo = __floats2bfloat162_rn(v[0], v[1]);
  const __nv_bfloat162 hi = __floats2bfloat162_rn(v[2], v[3]);
  uint2 u;
  u.x = *reinterpret_cast<const unsigned*>(&lo);
  u.y = *reinterpret_cast<const unsigned*>(&hi);
  *reinterpret_cast<uint2*>(p) = u;
}

// 4 consecutive elements from a staging slot (16- or 8-byte aligned)
__device__ __forceinline__ void ld4s(const float* p, float (&o)[4]) {
  const float4 v = *reinterpret_cast<const float4*>(p);
  o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
}
__device__ __forceinline__ void ld4s(const __nv_bfloat16* p, float (&o)[4]) {
  const uint2 v = *reinterpret_cast<const uint2*>(p);
  o[0] = __uint_as_float(v.x << 16); o[1] = __uint_as_float(v.x & 0xffff0000u);
  o[2] = __uint_as_float(v.y << 16); o[3] = __uint_as_float(v.y & 0xffff0000u);
}

__device__ __forceinline__ float win_val(const float* s, int i) { return s[i]; }
__device__ __forceinline__ float win_val(const __nv_bfloat16* s, int i) { return __bfloat162float(s[i]); }

// out[j] += (A x or A^T x) at rows r0 + 4a + j of column c0 + cl, for every
// separable term. st: taps of the forward factors in shared memory, row
// factors [t][w] then column factors [t][w] (tap k multiplies the pixel at
// offset dlo + k); the transposed blur takes them reversed. sx: the window,
// sz: TN * ZP floats. Each pass runs tap by tap over a register window, so
// one (broadcast) tap load feeds 8 or 4 FMAs and one window load w of them.
// Synchronises the block between the passes (and between terms).
template <int KW, typename Tw>
__device__ __forceinline__ void toep_conv(const ToepGeom& g, int w, int nterms, const float* st, bool tr,
                                          const Tw* sx, float* sz, float (&out)[4]) {
  const int lane = threadIdx.x, wid = threadIdx.y;
  const int tid = lane + 32 * wid;
  for (int t = 0; t < nterms; ++t) {
    // column pass: sz[c][r] = sum_k fc[k] x(box row r, box column c + k), for
    // every box row and the TN output columns; lanes run over rows, each
    // thread over 8 consecutive output columns
    {
      const float* fc = st + (size_t)(nterms + t) * w;
      const int q = wid & 3;
      for (int grp = wid >> 2; grp * 32 < g.RB; grp += 2) {
        const int r = grp * 32 + lane;
        if (r < g.RB) {
          float xv[KW + 7];
#pragma unroll
          for (int i = 0; i < KW + 7; ++i) xv[i] = i < w + 7 ? win_val(sx, (8 * q + i) * g.RB + r) : 0.f;
          float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
          for (int k = 0; k < KW; ++k) {
            if (k < w) {
              const float f = fc[tr ? w - 1 - k : k];
#pragma unroll
              for (int j = 0; j < 8; ++j) acc[j] = fmaf(f, xv[j + k], acc[j]);
            }
          }
#pragma unroll
          for (int j = 0; j < 8; ++j) sz[(8 * q + j) * g.ZP + r] = acc[j];
        }
      }
    }
    __syncthreads();
    // row pass: out[j] += sum_k fr[k] sz[cl][4a + j + s + k]
    {
      const float* fr = st + (size_t)t * w;
      const int a = tid & 7, cl = tid >> 3;
      const float* zs = sz + cl * g.ZP + 4 * a + g.s;
      float zv[KW + 3];
#pragma unroll
      for (int i = 0; i < KW + 3; ++i) zv[i] = i < w + 3 ? zs[i] : 0.f;
      float acc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
      for (int k = 0; k < KW; ++k) {
        if (k < w) {
          const float f = fr[tr ? w - 1 - k : k];
#pragma unroll
          for (int j = 0; j < 4; ++j) acc[j] = fmaf(f, zv[j + k], acc[j]);
        }
      }
#pragma unroll
      for (int j = 0; j < 4; ++j) out[j] += acc[j];
    }
    if (t + 1 < nterms) __syncthreads();
  }
}

template <typename Tw>
__device__ __forceinline__ void toep_conv_any(const ToepGeom& g, int w, int nterms, const float* st, bool tr,
                                              const Tw* sx, float* sz, float (&out)[4]) {
  if (w <= 8) toep_conv<8, Tw>(g, w, nterms, st, tr, sx, sz, out);
  else if (w <= 16) toep_conv<16, Tw>(g, w, nterms, st, tr, sx, sz, out);
  else if (w <= 24) toep_conv<24, Tw>(g, w, nterms, st, tr, sx, sz, out);
  else toep_conv<32, Tw>(g, w, nterms, st, tr, sx, sz, out);
}

// ---- standalone level-0 blur by the direct path ------------------------------
// Y = scale * A X (or A^T X) for float vectors; scale = 1 / sqrt(*nrm2) when
// nrm2 is given, and then xcopy (optional) receives the scaled input at the
// block's own pixels. Persistent over tiles with two window buffers: the
// copy of the tile after next is issued as soon as a buffer is free, so
// copies overlap the convolutions. A copy that does not land within
// TOEP_BLUR_LIMIT_NS sets *err and ends the block (after a bounded wait for
// any copy still in flight).
constexpr unsigned long long TOEP_BLUR_LIMIT_NS = 1000000000ull;

__host__ __device__ inline int toep_blur_smem_bytes(const ToepGeom& g) {
  return 128 + 2 * toep_win_bytes(g) + toep_z_bytes(g) + TOEP_TAP_BYTES;
}

__global__ void __launch_bounds__(256, 2)
    k_blur_direct(const __grid_constant__ CUtensorMap map, int m, int dlo, int w, int nterms,
                  const float* __restrict__ tp, int tr, float* __restrict__ Y, float scale, const double* nrm2,
                  float* __restrict__ xcopy, int* err) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t bar[2];
  const ToepGeom g = toep_geom(dlo, w);
  unsigned char* base = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 127) &
                                                         ~static_cast<uintptr_t>(127));
  unsigned char* win0 = base;
  unsigned char* win1 = base + toep_win_bytes(g);
  float* sz = reinterpret_cast<float*>(base + 2 * toep_win_bytes(g));
  float* stp = reinterpret_cast<float*>(base + 2 * toep_win_bytes(g) + toep_z_bytes(g));
  const int tid = threadIdx.x + 32 * threadIdx.y;
  if (nrm2) scale = (float)(1.0 / sqrt(*nrm2));
  for (int i = tid; i < 2 * nterms * w; i += 32 * TY) stp[i] = tp[i];
  if (tid == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
  }
  __syncthreads();
  const int nt = m / TM, ntiles = nt * nt;
  const unsigned bytes = (unsigned)(g.RB * g.CB * 4);
  // the window copies of this block's first two tiles
  unsigned pend = 0;   // (thread 0) buffers with a copy in flight
  if (tid == 0) {
    for (int q = 0; q < 2; ++q) {
      const int tile = blockIdx.x + q * (int)gridDim.x;
      if (tile >= ntiles) break;
      fence_proxy_async();
      mbar_arrive_expect_tx(&bar[q], bytes);
      tma_load_2d(q ? win1 : win0, &map, (tile % nt) * TM + g.f8, (tile / nt) * TN + dlo, &bar[q]);
      pend |= 1u << q;
    }
  }
  unsigned par = 0;    // parity bit of each buffer's next completion
  int q = 0;
  const int a = tid & 7, cl = tid >> 3;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, q ^= 1) {
    const int r0 = (tile % nt) * TM, c0 = (tile / nt) * TN;
    const bool ok = mbar_wait_bounded(&bar[q], (par >> q) & 1u, TOEP_BLUR_LIMIT_NS);
    if (__syncthreads_or(!ok)) {
      if (tid == 0) {
        atomicExch(err, 1);
        for (int b = 0; b < 2; ++b)
          if (pend & (1u << b)) mbar_wait_bounded(&bar[b], (par >> b) & 1u, TOEP_BLUR_LIMIT_NS);
      }
      return;
    }
    par ^= 1u << q;
    if (tid == 0) pend &= ~(1u << q);
    const float* sx = reinterpret_cast<const float*>(q ? win1 : win0);
    float out[4] = {0.f, 0.f, 0.f, 0.f};
    toep_conv_any<float>(g, w, nterms, stp, tr != 0, sx, sz, out);
    const int r = r0 + 4 * a, c = c0 + cl;
    const size_t i = r + (size_t)c * m;
    float o[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) o[j] = scale * out[j];
    st4(Y + i, o);
    if (xcopy) {
      const int wr = 4 * a - g.f8, wc = cl - dlo;
#pragma unroll
      for (int j = 0; j < 4; ++j) o[j] = scale * sx[wc * g.RB + wr + j];
      st4(xcopy + i, o);
    }
    __syncthreads();   // the window buffer and the intermediate are free again
    const int next = tile + 2 * (int)gridDim.x;
    if (tid == 0 && next < ntiles) {
      fence_proxy_async();
      mbar_arrive_expect_tx(&bar[q], bytes);
      tma_load_2d(q ? win1 : win0, &map, (next % nt) * TM + g.f8, (next / nt) * TN + dlo, &bar[q]);
      pend |= 1u << q;
    }
  }
}

}  // namespace db
