// libdeblur: host runtime and C-ABI (see include/deblur.h).
//
// A solve (Alg. 4) runs entirely on the device: the level hierarchy (bands of
// every Galerkin coarse operator, restricted right-hand sides), the outer
// solvers (Alg. 1-3), GCV (Sec. 3) and the transfers (Sec. 4.1). The host
// only sequences launches and reads one small status record per outer
// iteration (LSQR iteration count and the two RC norms) to take the stopping
// decision of Eq. (stop).
#include <cuda_runtime.h>
#include <cudaTypedefs.h>
#include <cstdio>
#include <cstring>
#include <cmath>
#include <string>
#include <vector>
#include <algorithm>
#include <type_traits>
#include <atomic>
#include <thread>
#include <memory>
#include <mutex>
#include <condition_variable>
#include <deque>
#include <map>
#include <chrono>
#include <functional>

#include "../../include/deblur.h"
#include "gcv.cuh"

using namespace db;

// ============================================================================
// error plumbing
// ============================================================================
struct DbError {
  db_status st;
  std::string msg;
};

#define CK(call)                                                                  \
  do {                                                                            \
    cudaError_t e_ = (call);                                                      \
    if (e_ != cudaSuccess) {                                                      \
      cudaGetLastError();                                                         \
      throw DbError{DB_ECUDA, std::string(#call) + " (deblur.cu:" + std::to_string(__LINE__) + "): " + \
                                  cudaGetErrorString(e_)};                                        \
    }                                                                             \
  } while (0)

#define REQUIRE(cond, text) \
  do { if (!(cond)) throw DbError{DB_EINVAL, text}; } while (0)

static thread_local std::string g_last_error;

// ============================================================================
// device arena owned by a context
// ============================================================================
struct Arena {
  char* base = nullptr;
  size_t cap = 0, off = 0;
  size_t budget = 0;
  Arena() = default;
  Arena(const Arena&) = delete;
  Arena& operator=(const Arena&) = delete;
  ~Arena() { if (base) cudaFree(base); }
  void reset() { off = 0; }
  void ensure(size_t bytes) {
    if (bytes <= cap) return;
    if (budget && bytes > budget) throw DbError{DB_ENOMEM, "workspace exceeds the context's HBM budget"};
    if (base) cudaFree(base);
    base = nullptr;
    cap = 0;
    if (cudaMalloc(&base, bytes) != cudaSuccess) {
      cudaGetLastError();
      throw DbError{DB_ENOMEM, "cudaMalloc of the workspace failed"};
    }
    cap = bytes;
  }
  template <typename X> X* take(size_t count) {
    size_t bytes = (count * sizeof(X) + 255) & ~size_t(255);
    if (off + bytes > cap) throw DbError{DB_ENOMEM, "workspace arena exhausted"};
    X* p = reinterpret_cast<X*>(base + off);
    off += bytes;
    return p;
  }
};

struct db_context {
  int device = 0;
  int nsm = 0;
  Arena arena;
  std::string err;
  db_stats stats{};
  std::atomic<uint64_t> n_launches{0}, n_gcv{0}, gcv_ns{0}, n_blur_direct{0};
  // launch-shape autotuner: size class -> chosen shape (see lsqr_launch)
  int autotune = 1;
  std::mutex tune_mu;
  std::map<uint64_t, int> tune_lsqr;
  int tuned(uint64_t key) {
    std::lock_guard<std::mutex> lk(tune_mu);
    auto it = tune_lsqr.find(key);
    return it == tune_lsqr.end() ? -1 : it->second;
  }
  void set_tuned(uint64_t key, int v) {
    std::lock_guard<std::mutex> lk(tune_mu);
    tune_lsqr[key] = v;
  }
  int profiling = 0;
  // factorisation of the last PSF (separable terms), reused while the PSF is unchanged
  std::vector<double> psf_key;
  double* psf_fr = nullptr;
  double* psf_fc = nullptr;
  int psf_nterms = 0;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
};

// Every kernel launch of the library is preceded by count_launch() so the
// context can report how many of its kernels ran.
static thread_local db_context* g_count_ctx = nullptr;
static inline void count_launch() {
  if (g_count_ctx) g_count_ctx->n_launches.fetch_add(1, std::memory_order_relaxed);
}
struct CountScope {
  db_context* prev;
  explicit CountScope(db_context* c) : prev(g_count_ctx) { g_count_ctx = c; }
  ~CountScope() { g_count_ctx = prev; }
};


static Filter make_filter(db_wavelet wv) {
  Filter f{};
  if (wv == DB_HAAR) {
    f.kappa = 2;
    f.h[0] = f.h[1] = std::sqrt(2.0) / 2.0;
  } else {
    const double s3 = std::sqrt(3.0), d = 4.0 * std::sqrt(2.0);
    f.kappa = 4;
    f.h[0] = (1 + s3) / d; f.h[1] = (3 + s3) / d; f.h[2] = (3 - s3) / d; f.h[3] = (1 - s3) / d;
  }
  return f;
}

// ---- tensor maps of the direct level-0 path ----------------------------------
// cuTensorMapEncodeTiled is reached through the runtime's driver entry point
// (no link against the driver library).
static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, []() {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    else
      cudaGetLastError();
  });
  return fn;
}

// Map of the m x m column-major image at `base` (elements of esz bytes) for
// the window box of toep_geom. The TMA rules are checked here, so a map that
// exists satisfies them: 16-byte aligned base, a row pitch that is a multiple
// of 16 bytes, an inner box extent that is a multiple of 16 bytes, box sides
// of at most 256 and a first box row (f8 + a multiple of the tile side) whose
// byte offset is a multiple of 16. Returns false when any rule fails or the
// encoder is unavailable (the level then keeps the band path).
static bool make_window_map(CUtensorMap* out, const void* base, int m, int esz, const ToepGeom& g) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!enc || !base || (esz != 2 && esz != 4)) return false;
  if ((reinterpret_cast<uintptr_t>(base) & 15) != 0) return false;
  if (((size_t)m * esz) % 16 != 0 || (g.RB * esz) % 16 != 0) return false;
  if (g.RB > 256 || g.CB > 256 || g.RB < 8) return false;
  if ((g.f8 * esz) % 16 != 0 || (TM * esz) % 16 != 0) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)m, (cuuint64_t)m};
  const cuuint64_t strides[1] = {(cuuint64_t)m * esz};
  const cuuint32_t box[2] = {(cuuint32_t)g.RB, (cuuint32_t)g.CB};
  const cuuint32_t estr[2] = {1, 1};
  const CUtensorMapDataType dt = esz == 2 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
  const CUresult r = enc(out, dt, 2, const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                         CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

// Dynamic shared-memory limit of a kernel (cudaFuncAttributeMaxDynamic-
// SharedMemorySize): a per-function, per-device setting that several host
// threads (the batched solver's GCV workers, other contexts) change while
// launching. It is only ever raised, under a lock, so a thread never lowers
// it below what another thread is about to launch with. Returns false when
// the device refuses the size.
static std::mutex g_smem_attr_mu;
static std::map<std::pair<int, const void*>, int> g_smem_attr;
static bool raise_smem_limit(const void* kfn, int bytes) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  std::lock_guard<std::mutex> lk(g_smem_attr_mu);
  int& cur = g_smem_attr[{dev, kfn}];
  if (bytes <= cur) return true;
  if (cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  cur = bytes;
  return true;
}
static void require_smem_limit(const void* kfn, int bytes) {
  if (!raise_smem_limit(kfn, bytes))
    throw DbError{DB_EINVAL, "kernel needs " + std::to_string(bytes) + " bytes of dynamic shared memory"};
}

static int grid_for(size_t n, int nsm, int per = 256) {
  size_t g = (n + per - 1) / per;
  size_t cap = (size_t)nsm * 8;
  if (g > cap) g = cap;
  if (g < 1) g = 1;
  return (int)g;
}

// Band-row cache of the LSQR kernel: on when every problem of the launch has
// a one-term (separable) blur and the cache (LSQR_TCACHE tiles x forward and
// transposed row and column bands) fits in 48 KB; sets the LsqrCtl fields and
// returns the extra dynamic shared memory in bytes.
template <typename Acc>
static int lsqr_band_cache(LsqrCtl& c, int tile_bytes, const BandOp<Acc>* ops, int nops) {
  c.band_cache = 0;
  c.band_pw = 0;
  c.cache_off = (tile_bytes + (int)sizeof(Acc) - 1) / (int)sizeof(Acc);
  int pw = 0;
  for (int i = 0; i < nops; ++i) {
    if (ops[i].nterms != 1) return 0;
    pw = std::max(pw, band_pitch(ops[i].w));
  }
  const int bytes = LSQR_TCACHE * 4 * TM * pw * (int)sizeof(Acc);
  if (nops < 1 || bytes > 48 * 1024) return 0;
  c.band_cache = 1;
  c.band_pw = pw;
  return c.cache_off * (int)sizeof(Acc) - tile_bytes + bytes;
}

// Launch shapes of the LSQR kernel the autotuner chooses between: the cap on
// resident blocks per SM (which sets how many tiles each block takes) and
// the band-row cache. Every shape computes the same result -- a tile's
// partial sums depend only on the tile and are added in tile order -- so the
// choice changes the time only.
struct LsqrShape {
  int per_sm_cap;
  int band_cache;
};
static const LsqrShape kLsqrShapes[4] = {{2, 1}, {2, 0}, {1, 1}, {1, 0}};

// Size class of an LSQR launch for the autotuner: storage size, tile count
// (power-of-two bucket), whether every blur has one term, widest band.
template <typename Acc>
static uint64_t lsqr_size_class(int elem_bytes, int ntiles, const BandOp<Acc>* ops, int nops) {
  int one = 1, w = 0;
  for (int i = 0; i < nops; ++i) {
    one &= ops[i].nterms == 1;
    w = std::max(w, ops[i].w);
  }
  int b = 0;
  while ((1 << b) < ntiles) ++b;
  return ((uint64_t)elem_bytes << 40) | ((uint64_t)b << 32) | ((uint64_t)one << 24) | (uint64_t)w;
}

template <typename T, typename Acc>
static void lsqr_launch(db_context* ctx, cudaStream_t st, const LsqrProb<T, Acc>* d_probs, LsqrCtl c, int ntiles,
                        int tile_bytes, const BandOp<Acc>* ops, int nops, LsqrShape shape) {
  int sm = tile_bytes;
  if (shape.band_cache) {
    sm += lsqr_band_cache<Acc>(c, tile_bytes, ops, nops);
  } else {
    c.band_cache = 0;
    c.band_pw = 0;
    c.cache_off = 0;
  }
  auto kfn = k_lsqr<T, Acc>;
  // the opt-in limit is raised on every launch, whatever the size: static
  // plus dynamic shared memory may pass the 48 KB default even when the
  // dynamic part alone does not
  require_smem_limit((const void*)kfn, sm);
  int per_sm = 0;
  CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kfn, 256, sm));
  if (per_sm < 1) throw DbError{DB_EINVAL, "LSQR kernel does not fit on an SM (" + std::to_string(sm) +
                                           " bytes of dynamic shared memory)"};
  per_sm = std::min(per_sm, shape.per_sm_cap);
  const int grid = std::max(1, std::min(ntiles, per_sm * ctx->nsm));
  void* args[] = {(void*)&d_probs, (void*)&c};
  count_launch();
  CK(cudaLaunchCooperativeKernel((const void*)kfn, dim3(grid), dim3(32, TY), args, sm, st));
}

// Runs one LSQR launch; on the first launch of a size class (autotune on)
// runs every shape on the same inputs, each a complete solve from the reset
// state, and keeps the fastest. Returns the device time of the launch whose
// results stay in the buffers (the last one run), in ms (profiling or tuning).
template <typename T, typename Acc, typename Reset>
static float lsqr_run(db_context* ctx, cudaStream_t st, const LsqrProb<T, Acc>* d_probs, const LsqrCtl& c,
                      int ntiles, int tile_bytes, const BandOp<Acc>* ops, int nops, GridBarrier* d_gb, Reset reset) {
  const uint64_t key = lsqr_size_class<Acc>((int)sizeof(T), ntiles, ops, nops);
  int choice = ctx->tuned(key);
  const bool tune = choice < 0 && ctx->autotune;
  if (choice < 0) choice = 0;
  const int first = tune ? 0 : choice, last = tune ? 3 : choice;
  float best = 1e30f, ms = 0.f;
  if ((tune || ctx->profiling) && !ctx->ev0) {
    std::lock_guard<std::mutex> lk(ctx->tune_mu);
    if (!ctx->ev0) {
      CK(cudaEventCreate(&ctx->ev1));
      CK(cudaEventCreate(&ctx->ev0));
    }
  }
  for (int s = first; s <= last; ++s) {
    reset();
    const bool timed = tune || ctx->profiling;
    if (timed) CK(cudaEventRecord(ctx->ev0, st));
    lsqr_launch<T, Acc>(ctx, st, d_probs, c, ntiles, tile_bytes, ops, nops, kLsqrShapes[s]);
    if (timed) {
      CK(cudaEventRecord(ctx->ev1, st));
      CK(cudaEventSynchronize(ctx->ev1));
      CK(cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1));
      GridBarrier gbh;
      CK(cudaMemcpyAsync(&gbh, d_gb, sizeof(gbh), cudaMemcpyDeviceToHost, st));
      CK(cudaStreamSynchronize(st));
      if (gbh.error) throw DbError{DB_ETIMEOUT, "LSQR grid barrier timed out"};
      if (ms < best) { best = ms; choice = s; }
    }
  }
  if (tune) ctx->set_tuned(key, choice);
  return ms;
}

// ============================================================================
// level hierarchy// ============================================================================
// level hierarchy
// ============================================================================
template <typename T>
struct Level {
  using Acc = typename Traits<T>::Acc;
  using X = typename Traits<T>::X;
  int m = 0;
  size_t n = 0;
  int dlo = 0, w = 0;
  double* Bd_r = nullptr;    // double bands [t][m][w]
  double* Bd_c = nullptr;
  Acc *br = nullptr, *bc = nullptr, *brT = nullptr, *bcT = nullptr;
  float* rho = nullptr;      // GCV symbol ratios [n]
  int ntaps = 0;             // level 0 of a sparse non-separable PSF: direct taps (BandOp)
  int* tap_pq = nullptr;
  Acc* tap_w = nullptr;
  int toep = 0;              // level 0 of a separable PSF: direct Toeplitz path of the LSQR passes
  Acc* tp = nullptr;         // its taps (row factors [t][w], column factors [t][w])
  CUtensorMap* tmaps = nullptr;   // window maps of v, uA, xa, xb (device)
  double* b64 = nullptr;     // right-hand side in double (levels that use the exact GCV)
  // vectors
  T* b = nullptr;
  X* xa = nullptr;           // outer iterate (two ping-pong buffers)
  X* xb = nullptr;
  T *uA = nullptr, *uLx = nullptr, *uLy = nullptr, *v = nullptr, *wv = nullptr;
  X* dlt = nullptr;          // LSQR correction
  T *a0x = nullptr, *a0y = nullptr, *a1x = nullptr, *a1y = nullptr;
  int ntiles_side() const { return (m + TM - 1) / TM; }
  BandOp<Acc> op(int nterms) const {
    BandOp<Acc> o;
    o.m = m; o.nterms = nterms; o.dlo = dlo; o.w = w;
    o.br = br; o.bc = bc; o.brT = brT; o.bcT = bcT;
    o.ntaps = ntaps; o.tap_pq = tap_pq; o.tap_w = tap_w;
    o.toep = toep; o.tp = tp;
    return o;
  }
};

static void coarse_band_shape(int m_c, int dlo, int w, int kappa, int* dlo2, int* w2) {
  // nonzero offsets of the coarse factor: [ceil((dlo-(kappa-1))/2), floor((dlo+w-1+kappa-1)/2)]
  int lo = (int)std::ceil((dlo - (kappa - 1)) / 2.0);
  int hi = (int)std::floor((dlo + w - 1 + kappa - 1) / 2.0);
  if (hi - lo + 1 >= m_c) { *dlo2 = -(m_c / 2); *w2 = m_c; }
  else { *dlo2 = lo; *w2 = hi - lo + 1; }
}

template <typename T>
struct Hierarchy {
  using Acc = typename Traits<T>::Acc;
  int nterms = 0, S = 0, levels = 0;
  std::vector<Level<T>> lv;
};

template <typename T>
__global__ void k_convert_in(size_t n, const double* __restrict__ x, T* __restrict__ y) {
  using Acc = typename Traits<T>::Acc;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    y[i] = store_cast<T, Acc>((Acc)x[i]);
}
template <typename T>
__global__ void k_convert_out(size_t n, const T* __restrict__ x, double* __restrict__ y) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    y[i] = (double)to_acc(x[i]);
}
template <typename T>
__global__ void k_fill(size_t n, T* __restrict__ y, double v) {
  using Acc = typename Traits<T>::Acc;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    y[i] = store_cast<T, Acc>((Acc)v);
}

// ============================================================================
// the solver for one storage type
// ============================================================================
// Device workspace of one GCV evaluation (Krylov basis, Gram matrices, the
// small problem). A batch shares a few of these among its problems.
template <typename Acc>
struct GcvBufs {
  Acc* gV = nullptr;
  Acc *gt = nullptr, *gz = nullptr, *gy = nullptr, *gatb = nullptr, *gdtc = nullptr, *gknext = nullptr;
  Acc *gcx = nullptr, *gcy = nullptr;
  double *gGA = nullptr, *gGD = nullptr, *ggA = nullptr, *ggD = nullptr, *gh = nullptr, *gwork = nullptr;
  double* gmdot_part = nullptr;
  double *gAd = nullptr, *gbA = nullptr, *gbD = nullptr, *gh2 = nullptr;
  double* gtrt = nullptr;             // symbol traces on the first selection grid
  size_t gwork_cap = 0;               // doubles in gwork
  float2* gpart2 = nullptr;
  size_t gpart2_cap = 0;
  float* gsk = nullptr;               // block partials of k_gram_dtd
  size_t gsk_blocks = 0;              // blocks they have room for
  int gkmax = 0;
  size_t gn = 0;
  // Krylov basis K_k(A^T A, A^T b) of the projected GCV, kept between calls on
  // the same level of the same solve (it depends on A and b only, not on the
  // weights or the shift): columns V_0..V_{kc_cols-1} with their G_A and g_A
  // entries, A^T b in gatb, the pending next direction in gt with its
  // squared norm in gpend (device).
  const void* kc_b = nullptr;
  uint64_t kc_epoch = 0;
  int kc_cols = 0;
  double kc_bnorm2 = 0.0, kc_atb2 = 0.0;
  double* gpend = nullptr;

  static size_t bytes(size_t n0, int kmax, int exact_max, int nsm) {
    size_t tot = n0 * sizeof(Acc) * (kmax + 9);
    tot += (size_t)kmax * kmax * sizeof(double) * 8 + (size_t)kmax * 4096 * sizeof(double);
    tot += (size_t)exact_max * exact_max * sizeof(double) + (size_t)kmax * 160 * sizeof(double);
    tot += (size_t)(2 * kmax + 4) * std::max<size_t>((n0 + 2047) / 2048, (size_t)4 * nsm) * 8;
    tot += sk_blocks(nsm) * SK_SLOTS * sizeof(float);
    return tot + 64 * 4096 + 1024;
  }

  static size_t sk_blocks(int nsm) { return (size_t)2 * nsm + 8; }

  void alloc(Arena& A, size_t n0, int kmax, int exact_max, int nsm) {
    gkmax = kmax;
    gn = n0;
    gV = A.take<Acc>((size_t)kmax * n0);
    gt = A.take<Acc>(n0); gz = A.take<Acc>(n0); gy = A.take<Acc>(n0);
    gatb = A.take<Acc>(n0); gdtc = A.take<Acc>(n0); gknext = A.take<Acc>(n0);
    gcx = A.take<Acc>(n0); gcy = A.take<Acc>(n0);
    gGA = A.take<double>((size_t)kmax * kmax);
    gGD = A.take<double>((size_t)kmax * kmax);
    ggA = A.take<double>(kmax);
    ggD = A.take<double>(kmax);
    gh = A.take<double>(kmax);
    // three projected selections side by side (batched IRLS steps), or one
    // selection of the largest basis (the exact mode's whole level)
    gwork_cap = std::max((size_t)3 * kmax * kmax + (7 + 2 * SEL_MAXPTS + 8) * (size_t)kmax, sel_work_doubles(kmax));
    gwork = A.take<double>(gwork_cap);
    gAd = A.take<double>((size_t)std::max(exact_max, 1) * std::max(exact_max, 1));
    gbA = A.take<double>(kmax);
    gbD = A.take<double>(kmax);
    gh2 = A.take<double>(kmax);
    gtrt = A.take<double>(SEL_MAXPTS);
    gpend = A.take<double>(1);
    kc_b = nullptr;
    kc_epoch = 0;
    kc_cols = 0;
    const size_t nch = std::max<size_t>((n0 + VCH_CHUNK - 1) / VCH_CHUNK, (size_t)4 * nsm);
    gpart2_cap = (size_t)(2 * kmax + 4) * nch;
    gpart2 = A.take<float2>(gpart2_cap);
    gmdot_part = A.take<double>((size_t)kmax * 256);
    gsk_blocks = sk_blocks(nsm);
    gsk = A.take<float>(gsk_blocks * SK_SLOTS);
  }
};

template <typename T>
struct Engine {
  using Acc = typename Traits<T>::Acc;
  using X = typename Traits<T>::X;
  db_context* ctx;
  cudaStream_t st;
  Hierarchy<T> H;
  db_opts o;
  db_gcv_opts go;
  Arena* arena = nullptr;            // null: the context's arena
  // scratch shared by all levels
  double* d_part = nullptr;
  size_t part_cap = 0;
  unsigned* d_cnt = nullptr;
  double* d_box = nullptr;           // small device mailbox
  GridBarrier* d_gb = nullptr;
  LsqrState* d_st = nullptr;
  LsqrCoef<Acc>* d_coef = nullptr;
  LsqrProb<T, Acc>* d_prob = nullptr;
  int* d_tile_prob = nullptr;
  // GCV workspace (owned or lent by a batch; see GcvBufs)
  Acc* gV = nullptr;
  Acc *gt = nullptr, *gz = nullptr, *gy = nullptr, *gatb = nullptr, *gdtc = nullptr, *gknext = nullptr;
  Acc *gcx = nullptr, *gcy = nullptr;
  double *gGA = nullptr, *gGD = nullptr, *ggA = nullptr, *ggD = nullptr, *gh = nullptr, *gwork = nullptr;
  double* gmdot_part = nullptr;
  double *gAd = nullptr, *gbA = nullptr, *gbD = nullptr, *gh2 = nullptr;
  double* gtrt = nullptr;
  size_t gwork_cap = 0;
  float2* gpart2 = nullptr;
  size_t gpart2_cap = 0;
  float* gsk = nullptr;
  size_t gsk_blocks = 0;
  int gkmax = 0;
  size_t gn = 0;

  GcvBufs<Acc>* gcur = nullptr;      // the buffers in use (for the Krylov cache)
  std::vector<Acc> host_taps;        // level-0 taps while their upload is in flight
  std::vector<int> host_tap_pq;
  std::vector<CUtensorMap> host_tmaps;   // level-0 window maps while their upload is in flight
  int* d_blur_err = nullptr;         // copy-timeout flag of the direct level-0 blur
  GcvBufs<Acc> own_bufs;
  uint64_t epoch = 0;                // unique per build (keys the Krylov cache)

  void adopt(GcvBufs<Acc>& b) {
    gcur = &b;
    gV = b.gV; gt = b.gt; gz = b.gz; gy = b.gy; gatb = b.gatb; gdtc = b.gdtc; gknext = b.gknext;
    gcx = b.gcx; gcy = b.gcy; gGA = b.gGA; gGD = b.gGD; ggA = b.ggA; ggD = b.ggD; gh = b.gh; gwork = b.gwork;
    gmdot_part = b.gmdot_part; gAd = b.gAd; gbA = b.gbA; gbD = b.gbD; gh2 = b.gh2; gtrt = b.gtrt; gwork_cap = b.gwork_cap; gpart2 = b.gpart2;
    gpart2_cap = b.gpart2_cap; gkmax = b.gkmax; gn = b.gn; gsk = b.gsk; gsk_blocks = b.gsk_blocks;
  }

  Engine(db_context* c, cudaStream_t s) : ctx(c), st(s) {}

  // ---------------------------------------------------------------- setup
  static int gram_dim(const db_gcv_opts& g) {
    return std::max(std::max(g.proj_dim_max, g.proj_dim), std::max(g.exact_max_pixels, 0)) + 2;
  }

  static size_t footprint_levels(int m, int levels, int S) {
    size_t tot = 0;
    for (int i = 0; i < levels; ++i) {
      int mi = m >> i;
      size_t n = (size_t)mi * mi;
      tot += n * (sizeof(T) * 16 + sizeof(X) * 3) + n * sizeof(float) + n * sizeof(double);
      tot += (size_t)mi * (S + 64) * (sizeof(double) * 2 + sizeof(Acc) * 4) * S + 4096;
      tot += (size_t)4 * S * m * 16;
      tot += 16384;   // direct-path taps and tensor maps
    }
    return tot + ((size_t)m * m / 1024 + 64) * 6 * sizeof(double) + 8 * 4096 + ((size_t)2 * S * S + S) * 8;
  }

  static size_t footprint(int m, int levels, int S, const db_gcv_opts& g) {
    return footprint_levels(m, levels, S) + GcvBufs<Acc>::bytes((size_t)m * m, gram_dim(g), g.exact_max_pixels, 160) +
           (16ull << 20);
  }

  void build(const double* psf_dev, int S, int m, int levels, db_wavelet wv, const double* b_dev, bool with_vectors,
             bool with_gcv = true) {
    Arena& A = arena ? *arena : ctx->arena;
    static std::atomic<uint64_t> build_counter{0};
    epoch = ++build_counter;
    d_blur_err = nullptr;
    H.S = S;
    H.levels = levels;
    H.lv.assign(levels, Level<T>());
    // PSF factorisation (rank-revealing one-sided Jacobi SVD), cached per PSF
    std::vector<double> key((size_t)S * S + 1);
    key[0] = (double)S;
    CK(cudaMemcpyAsync(key.data() + 1, psf_dev, (size_t)S * S * sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    const double* fr;
    const double* fc;
    int nterms = 0;
    if (ctx->psf_fr && key == ctx->psf_key) {
      fr = ctx->psf_fr;
      fc = ctx->psf_fc;
      nterms = ctx->psf_nterms;
    } else {
      if (ctx->psf_fr) { cudaFree(ctx->psf_fr); cudaFree(ctx->psf_fc); ctx->psf_fr = ctx->psf_fc = nullptr; }
      ctx->psf_key.clear();
      double *nfr = nullptr, *nfc = nullptr;
      CK(cudaMalloc(&nfr, (size_t)S * S * sizeof(double)));
      CK(cudaMalloc(&nfc, (size_t)S * S * sizeof(double)));
      ctx->psf_fr = nfr;
      ctx->psf_fc = nfc;
      double* wk = A.take<double>((size_t)2 * S * S + S);
      int* d_nt = A.take<int>(1);
      { count_launch(); k_psf_svd<<<1, 256, 0, st>>>(S, psf_dev, 1e-13, d_nt, nfr, nfc, wk); }
      CK(cudaGetLastError());
      CK(cudaMemcpyAsync(&nterms, d_nt, sizeof(int), cudaMemcpyDeviceToHost, st));
      CK(cudaStreamSynchronize(st));
      REQUIRE(nterms >= 1, "PSF is zero");
      ctx->psf_nterms = nterms;
      ctx->psf_key = key;
      fr = nfr;
      fc = nfc;
    }
    H.nterms = nterms;
    // non-zero taps of the PSF (column-major, psf[(p + R) + (q + R) S])
    std::vector<int> tpq;
    host_taps.clear();
    for (int q = -(S / 2); q <= S / 2; ++q)
      for (int p = -(S / 2); p <= S / 2; ++p) {
        const double v = key[1 + (p + S / 2) + (size_t)(q + S / 2) * S];
        if (v != 0.0) {
          tpq.push_back(((p + 128) << 8) | (q + 128));
          host_taps.push_back((Acc)v);
        }
      }
    host_tap_pq = tpq;
    const Filter f = make_filter(wv);
    const int kmax = gram_dim(go);
    for (int i = 0; i < levels; ++i) {
      Level<T>& L = H.lv[i];
      L.m = m >> i;
      L.n = (size_t)L.m * L.m;
      if (i == 0) { L.dlo = -(S / 2); L.w = S; }
      else coarse_band_shape(L.m, H.lv[i - 1].dlo, H.lv[i - 1].w, f.kappa, &L.dlo, &L.w);
      REQUIRE(L.w <= MAX_BAND, "coarse operator band too wide for the tile kernels");
      size_t nb = (size_t)nterms * L.m * L.w;
      L.Bd_r = A.take<double>(nb);
      L.Bd_c = A.take<double>(nb);
      L.br = A.take<Acc>(nb); L.bc = A.take<Acc>(nb); L.brT = A.take<Acc>(nb); L.bcT = A.take<Acc>(nb);
      const int gb = grid_for(nb, ctx->nsm);
      if (i == 0) {
        // a non-separable PSF with few non-zero taps (a motion blur) is
        // applied directly on level 0: fewer operations than its separable
        // terms (about nterms * 3 * S per pixel)
        const int nnz = (int)host_tap_pq.size();
        if (nterms > 1 && nnz < nterms * 2 * S && nnz <= MAX_TAPS && nnz <= TM * band_pitch(L.w)) {
          L.ntaps = nnz;
          L.tap_pq = A.take<int>(nnz);
          L.tap_w = A.take<Acc>(nnz);
          CK(cudaMemcpyAsync(L.tap_pq, host_tap_pq.data(), nnz * sizeof(int), cudaMemcpyHostToDevice, st));
          CK(cudaMemcpyAsync(L.tap_w, host_taps.data(), nnz * sizeof(Acc), cudaMemcpyHostToDevice, st));
        }
        { count_launch(); k_fine_bands_d<<<gb, 256, 0, st>>>(L.m, S, nterms, fr, L.Bd_r); }
        { count_launch(); k_fine_bands_d<<<gb, 256, 0, st>>>(L.m, S, nterms, fc, L.Bd_c); }
      } else {
        const Level<T>& P = H.lv[i - 1];
        { count_launch(); k_coarsen_bands<<<gb, 256, 0, st>>>(P.m, P.dlo, P.w, nterms, f, P.Bd_r, L.dlo, L.w, L.Bd_r); }
        { count_launch(); k_coarsen_bands<<<gb, 256, 0, st>>>(P.m, P.dlo, P.w, nterms, f, P.Bd_c, L.dlo, L.w, L.Bd_c); }
      }
      { count_launch(); k_transpose_band<Acc><<<gb, 256, 0, st>>>(L.m, L.dlo, L.w, nterms, L.Bd_r, L.br, L.brT); }
      { count_launch(); k_transpose_band<Acc><<<gb, 256, 0, st>>>(L.m, L.dlo, L.w, nterms, L.Bd_c, L.bc, L.bcT); }
      CK(cudaGetLastError());
      if (with_vectors) {
        const size_t n = L.n;
        L.rho = A.take<float>(n);
        double2* Kr = A.take<double2>((size_t)nterms * L.m);
        double2* Kc = A.take<double2>((size_t)nterms * L.m);
        const int g1 = grid_for((size_t)nterms * L.m, ctx->nsm);
        { count_launch(); k_band_dft<<<g1, 256, 0, st>>>(L.m, L.dlo, L.w, nterms, L.Bd_r, Kr); }
        { count_launch(); k_band_dft<<<g1, 256, 0, st>>>(L.m, L.dlo, L.w, nterms, L.Bd_c, Kc); }
        { count_launch(); k_symbol_rho<<<grid_for(n, ctx->nsm), 256, 0, st>>>(L.m, nterms, Kr, Kc, L.rho); }
        CK(cudaGetLastError());
        L.b = A.take<T>(n);
        L.xa = A.take<X>(n); L.xb = A.take<X>(n);
        L.uA = A.take<T>(n); L.uLx = A.take<T>(n); L.uLy = A.take<T>(n);
        L.v = A.take<T>(n); L.wv = A.take<T>(n); L.dlt = A.take<X>(n);
        L.a0x = A.take<T>(n); L.a0y = A.take<T>(n); L.a1x = A.take<T>(n); L.a1y = A.take<T>(n);
      }
      if (i == 0) setup_direct(L, A, nterms, S, with_vectors);
    }
    if (with_vectors && b_dev) {
      const size_t n0 = H.lv[0].n;
      // double copy of b on every level small enough for the exact GCV
      // (restricted in double from the input)
      const double* bprev = b_dev;
      for (int i = 0; i < levels; ++i) {
        Level<T>& L = H.lv[i];
        if (i > 0) {
          double* bi = A.take<double>(L.n);
          { count_launch(); k_restrict<double><<<grid_for(L.n, ctx->nsm), 256, 0, st>>>(H.lv[i - 1].m, f, bprev, bi); }
          bprev = bi;
        }
        if ((long long)L.n <= (long long)go.exact_max_pixels) L.b64 = const_cast<double*>(bprev);
      }
      { count_launch(); k_convert_in<T><<<grid_for(n0, ctx->nsm), 256, 0, st>>>(n0, b_dev, H.lv[0].b); }
      for (int i = 1; i < levels; ++i) {
        const Level<T>& P = H.lv[i - 1];
        { count_launch(); k_restrict<T><<<grid_for(H.lv[i].n, ctx->nsm), 256, 0, st>>>(P.m, f, P.b, H.lv[i].b); }
      }
      CK(cudaGetLastError());
    }
    // shared scratch
    const size_t n0 = (size_t)m * m;
    size_t ntiles = 0;
    for (auto& L : H.lv) ntiles = std::max(ntiles, (size_t)L.ntiles_side() * L.ntiles_side());
    part_cap = std::max<size_t>(ntiles * 6 + 64, 8192);   // LSQR tile partials, two phase buffers
    d_part = A.take<double>(part_cap);
    d_cnt = A.take<unsigned>(64);
    d_box = A.take<double>(64);
    d_gb = A.take<GridBarrier>(1);
    d_st = A.take<LsqrState>(1);
    d_coef = A.take<LsqrCoef<Acc>>(1);
    d_prob = A.take<LsqrProb<T, Acc>>(1);
    d_tile_prob = A.take<int>(ntiles + 1);
    CK(cudaMemsetAsync(d_cnt, 0, 64 * sizeof(unsigned), st));
    CK(cudaMemsetAsync(d_gb, 0, sizeof(GridBarrier), st));
    if (with_vectors && with_gcv) {
      own_bufs.alloc(A, n0, kmax, go.exact_max_pixels, ctx->nsm);
      adopt(own_bufs);
    }
  }

  // Direct Toeplitz path of the level-0 LSQR passes (toep.cuh): float
  // working precision, a separable PSF (no direct taps) of odd side <= 32,
  // a side of at least 64 (every tile full, the middle row of a band holds
  // all taps), and tensor maps that pass the TMA rules. Otherwise the level
  // keeps the band path.
  void setup_direct(Level<T>& L, Arena& A, int nterms, int S, bool with_vectors) {
    L.toep = 0;
    L.tmaps = nullptr;
    if (!std::is_same<Acc, float>::value || !o.fine_direct || L.ntaps > 0) return;
    if ((S & 1) == 0 || S > TOEP_MAX_W || L.m < 64 || L.m % TM != 0 || L.w != S || L.dlo != -(S / 2)) return;
    if (nterms * S > TOEP_MAX_TAPS) return;
    if (!d_blur_err) {
      d_blur_err = A.take<int>(1);
      CK(cudaMemsetAsync(d_blur_err, 0, sizeof(int), st));
    }
    const ToepGeom g = toep_geom(L.dlo, L.w);
    host_tmaps.assign(4, CUtensorMap{});
    // the LSQR window maps (levels with vectors); without them the level
    // still applies the standalone blur directly
    if (with_vectors && make_window_map(&host_tmaps[0], L.v, L.m, (int)sizeof(T), g) &&
        make_window_map(&host_tmaps[1], L.uA, L.m, (int)sizeof(T), g) &&
        make_window_map(&host_tmaps[2], L.xa, L.m, (int)sizeof(X), g) &&
        make_window_map(&host_tmaps[3], L.xb, L.m, (int)sizeof(X), g)) {
      L.tmaps = A.take<CUtensorMap>(4);
      CK(cudaMemcpyAsync(L.tmaps, host_tmaps.data(), 4 * sizeof(CUtensorMap), cudaMemcpyHostToDevice, st));
    }
    // taps: the middle row of each band (an interior row, where the zero
    // boundary cuts nothing)
    L.tp = A.take<Acc>((size_t)2 * nterms * S);
    const size_t pitch = (size_t)L.m * S * sizeof(Acc);
    CK(cudaMemcpy2DAsync(L.tp, S * sizeof(Acc), L.br + (size_t)(L.m / 2) * S, pitch, S * sizeof(Acc), nterms,
                         cudaMemcpyDeviceToDevice, st));
    CK(cudaMemcpy2DAsync(L.tp + (size_t)nterms * S, S * sizeof(Acc), L.bc + (size_t)(L.m / 2) * S, pitch,
                         S * sizeof(Acc), nterms, cudaMemcpyDeviceToDevice, st));
    L.toep = 1;
  }

  // Window maps of a problem's LSQR launch on a level with the direct path;
  // an x0 that is neither of the level's iterates turns the path off.
  static void set_direct(LsqrProb<T, Acc>& P, const Level<T>& L, const X* x0) {
    if (!P.op.toep) return;
    if (!L.tmaps) { P.op.toep = 0; return; }
    P.tm_v = L.tmaps + 0;
    P.tm_u = L.tmaps + 1;
    P.tm_x0 = x0 == L.xa ? L.tmaps + 2 : x0 == L.xb ? L.tmaps + 3 : nullptr;
    if (x0 && !P.tm_x0) P.op.toep = 0;
  }

  // ---------------------------------------------------------------- operators
  int smem_bytes(const BandOp<Acc>& op) const {
    TileGeom g = tile_geom(op, false), gt = tile_geom(op, true);
    int b = std::max(tile_smem_elems(g.H, g.w), tile_smem_elems(gt.H, gt.w)) * (int)sizeof(Acc);
    if (op.toep) b = std::max(b, toep_smem_bytes(toep_geom(op.dlo, op.w)));
    return b;
  }

  // Level-0 blur of float vectors by the direct path (k_blur_direct); false
  // when the level or the vector does not qualify (the caller then uses the
  // band form).
  bool blur_direct(const Level<T>& L, bool tr, const void* x, void* y, float scale, const double* nrm2, void* xcopy) {
    if (!std::is_same<Acc, float>::value || !L.toep || !d_blur_err) return false;
    const ToepGeom g = toep_geom(L.dlo, L.w);
    CUtensorMap map;
    if (!make_window_map(&map, x, L.m, 4, g)) return false;
    if ((reinterpret_cast<uintptr_t>(y) & 15) || (reinterpret_cast<uintptr_t>(xcopy) & 15)) return false;
    const int sm = toep_blur_smem_bytes(g);
    if (sm > 48 * 1024) require_smem_limit((const void*)k_blur_direct, sm);
    const int nt = L.ntiles_side();
    const int grid = std::min(nt * nt, 2 * ctx->nsm);
    count_launch();
    ctx->n_blur_direct.fetch_add(1, std::memory_order_relaxed);
    k_blur_direct<<<grid, dim3(32, TY), sm, st>>>(map, L.m, L.dlo, L.w, H.nterms, reinterpret_cast<const float*>(L.tp),
                                                 tr ? 1 : 0, static_cast<float*>(y), scale, nrm2,
                                                 static_cast<float*>(xcopy), d_blur_err);
    CK(cudaGetLastError());
    return true;
  }

  // Reads and clears the direct blur's copy-timeout flag.
  void check_blur_err() {
    if (!d_blur_err) return;
    int e = 0;
    CK(cudaMemcpyAsync(&e, d_blur_err, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (e) {
      CK(cudaMemsetAsync(d_blur_err, 0, sizeof(int), st));
      throw DbError{DB_ETIMEOUT, "a window copy of the level-0 blur did not complete"};
    }
  }

  void blur(const Level<T>& L, bool tr, const Acc* x, Acc* y, Acc scale = Acc(1)) {
    if (blur_direct(L, tr, x, y, (float)scale, nullptr, nullptr)) return;
    BandOp<Acc> op = L.op(H.nterms);
    const int sm = smem_bytes(op);
    if (sm > 48 * 1024) require_smem_limit((const void*)k_blur<Acc, Acc>, sm);
    const int nt = L.ntiles_side();
    const int grid = std::min(nt * nt, ctx->nsm * 8);
    { count_launch(); k_blur<Acc, Acc><<<grid, dim3(32, TY), sm, st>>>(op, tr ? 1 : 0, x, y, scale); }
    CK(cudaGetLastError());
  }

  void blur_T(const Level<T>& L, bool tr, const T* x, T* y) {
    if (std::is_same<T, float>::value && blur_direct(L, tr, x, y, 1.f, nullptr, nullptr)) return;
    BandOp<Acc> op = L.op(H.nterms);
    const int sm = smem_bytes(op);
    if (sm > 48 * 1024) require_smem_limit((const void*)k_blur<T, Acc>, sm);
    const int nt = L.ntiles_side();
    const int grid = std::min(nt * nt, ctx->nsm * 8);
    { count_launch(); k_blur<T, Acc><<<grid, dim3(32, TY), sm, st>>>(op, tr ? 1 : 0, x, y, Acc(1)); }
    CK(cudaGetLastError());
  }

  double dot(size_t n, const Acc* x, const Acc* y) {
    const int g = grid_for(n, ctx->nsm);
    { count_launch(); k_dot<Acc, Acc><<<g, 256, 0, st>>>(n, x, y, d_part, d_cnt + 8, d_box + 8); }
    CK(cudaGetLastError());
    double v;
    CK(cudaMemcpyAsync(&v, d_box + 8, sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    return v;
  }
  template <typename X>
  void dot_dev(size_t n, const X* x, const X* y, double* out) {
    const int g = grid_for(n, ctx->nsm);
    { count_launch(); k_dot<X, X><<<g, 256, 0, st>>>(n, x, y, d_part, d_cnt + 9, out); }
    CK(cudaGetLastError());
  }

  // ---------------------------------------------------------------- LSQR
  int lsqr(const Level<T>& L, int solver, double gamma, const X* x0, int* stop_out = nullptr) {
    LsqrProb<T, Acc> P{};
    P.op = L.op(H.nterms);
    P.m = L.m;
    P.solver = solver;
    P.gamma = gamma;
    P.sg = (Acc)std::sqrt(gamma);
    P.b = L.b;
    P.x0 = x0;
    P.a0x = L.a0x; P.a0y = L.a0y; P.a1x = L.a1x; P.a1y = L.a1y;
    P.uA = L.uA; P.uLx = L.uLx; P.uLy = L.uLy; P.v = L.v; P.w = L.wv; P.dlt = L.dlt;
    P.nt = L.ntiles_side();
    P.ntiles = P.nt * P.nt;
    P.tile_begin = 0;
    set_direct(P, L, x0);
    if (P.op.toep) ctx->stats.lsqr_direct_solves++;
    CK(cudaMemcpyAsync(d_prob, &P, sizeof(P), cudaMemcpyHostToDevice, st));
    std::vector<int> tp(P.ntiles, 0);
    CK(cudaMemcpyAsync(d_tile_prob, tp.data(), sizeof(int) * tp.size(), cudaMemcpyHostToDevice, st));
    LsqrCtl c;
    c.atol = o.lsqr_atol; c.btol = o.lsqr_btol; c.conlim = o.lsqr_conlim; c.maxit = o.lsqr_maxit;
    c.nprob = 1; c.ntiles = P.ntiles;
    c.tile_prob = d_tile_prob; c.part = d_part; c.cnt = d_cnt; c.st = d_st; c.gb = d_gb; c.coef = d_coef;
    c.limit_ns = (unsigned long long)o.barrier_timeout_us * 1000ull;
    auto reset = [&]() {
      CK(cudaMemsetAsync(d_st, 0, sizeof(LsqrState), st));
      CK(cudaMemsetAsync(d_coef, 0, sizeof(LsqrCoef<Acc>), st));
      CK(cudaMemsetAsync(d_cnt, 0, sizeof(unsigned), st));
      CK(cudaMemsetAsync(d_gb, 0, sizeof(GridBarrier), st));
    };
    const float lsqr_ms = lsqr_run<T, Acc>(ctx, st, d_prob, c, P.ntiles, smem_bytes(P.op), &P.op, 1, d_gb, reset);
    LsqrState S;
    GridBarrier gbh;
    CK(cudaMemcpyAsync(&S, d_st, sizeof(S), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(&gbh, d_gb, sizeof(gbh), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (gbh.error) throw DbError{DB_ETIMEOUT, "LSQR grid barrier timed out"};
    if (stop_out) *stop_out = S.stop;
    ctx->stats.lsqr_launches++;
    const double pix = (double)(S.its + 1) * (double)L.n;
    if (solver == DB_IRLS) ctx->stats.lsqr_pixel_iters_irls += pix;
    else ctx->stats.lsqr_pixel_iters_other += pix;
    if (ctx->profiling) ctx->stats.lsqr_ms += lsqr_ms;
    if (!H.lv.empty() && &L == &H.lv[0]) {
      ctx->stats.lsqr_fine_launches++;
      if (solver == DB_IRLS) ctx->stats.lsqr_fine_pixel_iters_irls += pix;
      else ctx->stats.lsqr_fine_pixel_iters_other += pix;
      if (ctx->profiling) ctx->stats.lsqr_fine_ms += lsqr_ms;
    }
    return S.its;
  }

  // ---------------------------------------------------------------- GCV
  void mdot(size_t n, int nvec, const Acc* V, const Acc* y, double* out, int ostride) {
    int nch = (int)std::min<size_t>(256, (n + 2047) / 2048);
    nch = std::max(nch, 1);
    { count_launch(); k_mdot<Acc><<<dim3(nch, nvec), 256, 0, st>>>(n, nvec, V, n, y, gmdot_part); }
    { count_launch(); k_mdot_reduce<<<(nvec + 7) / 8, 256, 0, st>>>(nvec, nch, gmdot_part, out, ostride); }
    CK(cudaGetLastError());
  }
  void maxpy(size_t n, int nvec, const Acc* V, const double* h, int hstride, Acc* y) {
    { count_launch(); k_maxpy<Acc><<<grid_for(n, ctx->nsm), 256, 0, st>>>(n, nvec, V, n, h, hstride, y); }
    CK(cudaGetLastError());
  }

  // column j of the Gram matrices for basis vector V_j (all V_0..V_j present)
  void gram_column(const Level<T>& L, int j, const T* wx, const T* wy, bool has_c) {
    const size_t n = L.n;
    const int ld = gkmax;
    Acc* vj = gV + (size_t)j * n;
    blur(L, false, vj, gz);
    blur(L, true, gz, gt);
    { count_launch(); k_DtD<Acc, T><<<grid_for(n, ctx->nsm), 256, 0, st>>>(L.m, vj, wx, wy, gy); }
    CK(cudaGetLastError());
    // G[i][j] for i <= j stored at G[i*ld + j]
    mdot(n, j + 1, gV, gt, gGA + j, ld);
    mdot(n, j + 1, gV, gy, gGD + j, ld);
    mdot(n, 1, vj, gatb, ggA + j, 1);
    if (has_c) mdot(n, 1, vj, gdtc, ggD + j, 1);
    else CK(cudaMemsetAsync(ggD + j, 0, sizeof(double), st));
  }

  // Selections (k_gcv_select, one block each, at most three) in one launch;
  // in projected mode the symbol traces of the first grid (the same for all)
  // come from one many-block pass (k_trace_table) beforehand. Returns gamma
  // of each selection.
  std::vector<double> select_multi(GcvSelectArgs* as, int na) {
    REQUIRE(na >= 1 && na <= 3, "one to three selections per launch");
    const GcvSelectArgs& f = as[0];
    const double* tab = nullptr;
    if (!f.exact && f.rho && f.npts >= 3) {
      const int npts = std::min(f.npts, SEL_MAXPTS);
      int nb = (int)std::min<size_t>(((size_t)f.npix + TRT_CHUNK - 1) / TRT_CHUNK, (size_t)2 * ctx->nsm);
      nb = std::max(nb, 1);
      if ((size_t)npts * nb <= gpart2_cap) {
        { count_launch(); k_trace_table<<<nb, 256, 0, st>>>(f.rho, f.npix, f.s, f.lo, f.hi, npts, gpart2, d_cnt + 24,
                                                            gtrt); }
        CK(cudaGetLastError());
        tab = gtrt;
      }
    }
    int kmax = 0;
    for (int i = 0; i < na; ++i) {
      as[i].trace_tab = tab;
      kmax = std::max(kmax, as[i].kk);
      REQUIRE(as[i].work >= gwork && as[i].work + sel_work_doubles(as[i].kk) <= gwork + gwork_cap,
              "GCV selection workspace too small");
    }
    bool cluster = true;
    for (int i = 0; i < na; ++i) cluster = cluster && !as[i].exact && as[i].kk <= SCL_MAXK;
    if (cluster) cluster = launch_select_cluster(as, na, kmax);
    if (!cluster) {
      const size_t sm = sel_smem_bytes(kmax);
      require_smem_limit((const void*)k_gcv_select, (int)sm);
      { count_launch(); k_gcv_select<<<na, SEL_THREADS, sm, st>>>(as[0], as[na > 1 ? 1 : 0], as[na > 2 ? 2 : 0]); }
      CK(cudaGetLastError());
    }
    std::vector<double> g(na);
    for (int i = 0; i < na; ++i) CK(cudaMemcpyAsync(&g[i], as[i].out, sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    return g;
  }
  double select(GcvSelectArgs a) { return select_multi(&a, 1)[0]; }

  // One cluster of SCL_NC CTAs per selection (k_gcv_select_cl). Returns false
  // (nothing launched) when the device cannot hold such a cluster.
  bool launch_select_cluster(GcvSelectArgs* as, int na, int kmax) {
    const size_t sm = scl_layout(kmax).total * sizeof(double);
    if (!raise_smem_limit((const void*)k_gcv_select_cl, (int)sm)) return false;
    // the last (largest) selection on a cluster of its own; with three, the
    // two smaller ones share a second cluster, one after the other
    const int ncl = na == 3 ? 2 : na;
    const unsigned plan = na == 3 ? (0x4u | (0x3u << 4)) : (na == 2 ? (0x1u | (0x2u << 4)) : 0x1u);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(SCL_NC * ncl);
    cfg.blockDim = dim3(SCL_THREADS);
    cfg.dynamicSmemBytes = sm;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = SCL_NC;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int nclusters = 0;
    if (cudaOccupancyMaxActiveClusters(&nclusters, k_gcv_select_cl, &cfg) != cudaSuccess || nclusters < 1) {
      cudaGetLastError();
      return false;
    }
    count_launch();
    CK(cudaLaunchKernelEx(&cfg, k_gcv_select_cl, as[0], as[na > 1 ? 1 : 0], as[na > 2 ? 2 : 0], plan));
    return true;
  }

  double gcv(const Level<T>& L, int solver, bool weighted, bool shifted) {
    if (go.gamma_fixed > 0) return go.gamma_fixed;
    if (!ctx->profiling) return gcv_impl(L, solver, weighted, shifted);
    const auto t0 = std::chrono::steady_clock::now();
    const double g = gcv_impl(L, solver, weighted, shifted);
    ctx->gcv_ns.fetch_add((uint64_t)std::chrono::duration_cast<std::chrono::nanoseconds>(
                              std::chrono::steady_clock::now() - t0).count(), std::memory_order_relaxed);
    return g;
  }

  double gcv_impl(const Level<T>& L, int solver, bool weighted, bool shifted) {
    ctx->n_gcv.fetch_add(1, std::memory_order_relaxed);
    const size_t n = L.n;
    const int m = L.m;
    const int ld = gkmax;
    const int gsz = grid_for(n, ctx->nsm);
    const T* wx = weighted ? L.a0x : nullptr;
    const T* wy = weighted ? L.a0y : nullptr;
    // A^T b, ||b||^2 (kept with the Krylov basis of the projected mode)
    const bool fused = std::is_same<Acc, float>::value && (long long)n > (long long)go.exact_max_pixels;
    const bool kc_hit = fused && gcur && gcur->kc_cols > 0 && gcur->kc_b == (const void*)L.b &&
                        gcur->kc_epoch == epoch;
    // every other path writes the buffers the cache lives in (G_A, A^T b)
    if (!fused && gcur) { gcur->kc_b = nullptr; gcur->kc_cols = 0; }
    double bnorm2, atb2;
    if (kc_hit) {
      bnorm2 = gcur->kc_bnorm2;
      atb2 = gcur->kc_atb2;
    } else {
      { count_launch(); k_to_acc<T, Acc><<<gsz, 256, 0, st>>>(n, L.b, (const T*)nullptr, gz); }
      CK(cudaGetLastError());
      bnorm2 = dot(n, gz, gz);
      blur(L, true, gz, gatb);
      atb2 = dot(n, gatb, gatb);
    }
    // D^T c
    bool has_c = false;
    if (shifted) {
      { count_launch(); k_to_acc<T, Acc><<<gsz, 256, 0, st>>>(n, L.a0x, solver == 2 ? L.a1x : nullptr, gcx); }
      { count_launch(); k_to_acc<T, Acc><<<gsz, 256, 0, st>>>(n, L.a0y, solver == 2 ? L.a1y : nullptr, gcy); }
      { count_launch(); k_Lt_w<Acc, T><<<gsz, 256, 0, st>>>(m, gcx, gcy, (const T*)nullptr, (const T*)nullptr, gdtc); }
      CK(cudaGetLastError());
      has_c = dot(n, gdtc, gdtc) > 0.0;
    }
    double s = 1.0;
    if (weighted) {
      double* box = d_box + 16;
      dot_dev<T>(n, L.a0x, L.a0x, box);
      dot_dev<T>(n, L.a0y, L.a0y, box + 1);
      double h2[2];
      CK(cudaMemcpyAsync(h2, box, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
      CK(cudaStreamSynchronize(st));
      s = (h2[0] + h2[1]) / (2.0 * m * (m - 1));
    }
    if ((long long)n <= (long long)go.exact_max_pixels) {
      // exact mode: dense pair, exact trace
      const int nn = (int)n;
      const int g2 = grid_for(n * n, ctx->nsm);
      { count_launch(); k_dense_blur<<<g2, 256, 0, st>>>(m, H.nterms, L.dlo, L.w, L.Bd_r, L.Bd_c, gAd); }
      { count_launch(); k_gram_dense<<<g2, 256, 0, st>>>(nn, gAd, gGA, ld); }
      { count_launch(); k_dense_DtD<T><<<g2, 256, 0, st>>>(m, wx, wy, gGD, ld); }
      // A^T b, ||b||^2 and D^T c in double: the exact pencil of a tiny level is
      // numerically singular and amplifies any rounding of these
      const double* bd = L.b64;
      if (!bd) {
        { count_launch(); k_diff_to_double<T><<<gsz, 256, 0, st>>>(n, L.b, (const T*)nullptr, gh2); }
        bd = gh2;
      }
      { count_launch(); k_dense_matvecT<<<grid_for(n, ctx->nsm), 256, 0, st>>>(nn, gAd, bd, gbA); }
      dot_dev<double>(n, bd, bd, d_box + 30);
      double bnorm2_e = 0.0;
      CK(cudaMemcpyAsync(&bnorm2_e, d_box + 30, sizeof(double), cudaMemcpyDeviceToHost, st));
      CK(cudaStreamSynchronize(st));
      if (has_c) {
        double* cxd = gmdot_part;
        double* cyd = gmdot_part + n;
        { count_launch(); k_diff_to_double<T><<<gsz, 256, 0, st>>>(n, L.a0x, solver == 2 ? L.a1x : nullptr, cxd); }
        { count_launch(); k_diff_to_double<T><<<gsz, 256, 0, st>>>(n, L.a0y, solver == 2 ? L.a1y : nullptr, cyd); }
        { count_launch(); k_Lt_w<double, T><<<gsz, 256, 0, st>>>(m, cxd, cyd, (const T*)nullptr, (const T*)nullptr, gbD); }
      } else {
        CK(cudaMemsetAsync(gbD, 0, n * sizeof(double), st));
      }
      CK(cudaGetLastError());
      GcvSelectArgs a;
      a.kk = nn; a.ld = ld; a.GA = gGA; a.GD = gGD; a.gA = gbA; a.gD = gbD; a.kshift = -1;
      a.bnorm2 = bnorm2_e; a.n = (double)n; a.s = 1.0; a.rho = L.rho; a.npix = nn; a.exact = 1;
      a.lo = go.log10_gamma_lo; a.hi = go.log10_gamma_hi; a.tolx = go.refine_tol_log10;
      a.npts = go.grid_points; a.max_ext = 2; a.work = gwork; a.out = d_box + 24;
      return select(a);
    }
    if constexpr (std::is_same<Acc, float>::value) {
      return gcv_projected_fused(L, wx, wy, has_c, s, bnorm2, atb2, kc_hit);
    } else {
    // v_0 (double working precision: multi-launch path)
    CK(cudaMemcpyAsync(d_box + 20, &atb2, sizeof(double), cudaMemcpyHostToDevice, st));
    { count_launch(); k_scale_inv_sqrt<Acc><<<gsz, 256, 0, st>>>(n, gatb, d_box + 20, gV); }
    CK(cudaGetLastError());
    const double dtc_norm2 = has_c ? dot(n, gdtc, gdtc) : 0.0;
    int nK = 1;            // Krylov vectors materialised in gV
    int cols = 0;          // Krylov columns computed
    bool pending = false;  // gknext holds an unnormalised next Krylov vector
    bool broke = false;
    const int kcap = (int)std::min<size_t>((size_t)go.proj_dim_max, n);
    int kdim = std::min<int>(go.proj_dim, kcap);
    double gamma_prev = -1.0, gamma = 0.0;
    const bool check_breakdown = n <= 4096;
    for (;;) {
      // extend the Krylov basis to kdim vectors with their Gram columns
      while (cols < kdim && !broke) {
        if (cols == nK) {
          if (!pending) break;
          { count_launch(); k_scale_inv_sqrt<Acc><<<gsz, 256, 0, st>>>(n, gknext, d_box + 21, gV + (size_t)nK * n); }
          CK(cudaGetLastError());
          ++nK;
          pending = false;
        }
        const int j = cols;
        gram_column(L, j, wx, wy, has_c);
        ++cols;
        if (cols < kdim || cols < kcap) {
          // next direction: t = A^T A v_j orthogonalised against V_0..V_j, twice
          // (first pass reuses the Gram column: G_A[i][j] = V_i . t)
          CK(cudaMemcpyAsync(gknext, gt, n * sizeof(Acc), cudaMemcpyDeviceToDevice, st));
          maxpy(n, j + 1, gV, gGA + j, ld, gknext);
          mdot(n, j + 1, gV, gknext, gh, 1);
          maxpy(n, j + 1, gV, gh, 1, gknext);
          dot_dev<Acc>(n, gknext, gknext, d_box + 21);
          pending = true;
          if (check_breakdown) {
            double nt2;
            CK(cudaMemcpyAsync(&nt2, d_box + 21, sizeof(double), cudaMemcpyDeviceToHost, st));
            CK(cudaStreamSynchronize(st));
            if (std::sqrt(nt2) <= 1e-12 * std::sqrt(atb2)) { broke = true; pending = false; }
          }
        }
      }
      int kk = cols;
      // shift direction orth(D^T c) in slot kk
      if (has_c) {
        Acc* vc = gV + (size_t)kk * n;
        CK(cudaMemcpyAsync(vc, gdtc, n * sizeof(Acc), cudaMemcpyDeviceToDevice, st));
        for (int pass = 0; pass < 2; ++pass) {
          mdot(n, kk, gV, vc, gh, 1);
          maxpy(n, kk, gV, gh, 1, vc);
        }
        const double nc2 = dot(n, vc, vc);
        if (std::sqrt(nc2) > 1e-12 * std::sqrt(dtc_norm2)) {
          CK(cudaMemcpyAsync(d_box + 22, &nc2, sizeof(double), cudaMemcpyHostToDevice, st));
          { count_launch(); k_scale_inv_sqrt<Acc><<<gsz, 256, 0, st>>>(n, vc, d_box + 22, vc); }
          CK(cudaGetLastError());
          gram_column(L, kk, wx, wy, true);
          ++kk;
        }
      }
      // small problem + selection
      GcvSelectArgs a;
      a.kk = kk; a.ld = ld; a.GA = gGA; a.GD = gGD; a.gA = ggA; a.gD = ggD; a.kshift = -1;
      a.bnorm2 = bnorm2; a.n = (double)n; a.s = s; a.rho = L.rho; a.npix = (int)n; a.exact = 0;
      a.lo = go.log10_gamma_lo; a.hi = go.log10_gamma_hi; a.tolx = go.refine_tol_log10;
      a.npts = go.grid_points; a.max_ext = 2; a.work = gwork; a.out = d_box + 24;
      gamma = select(a);
      if (gamma_prev > 0 && std::fabs(gamma - gamma_prev) <= 1e-3 * gamma_prev) return gamma;
      if (2 * kdim > kcap || kdim >= (int)n || broke) return gamma;
      gamma_prev = gamma;
      kdim *= 2;
    }
    }
  }

  // Projected GCV with the fused Krylov kernels (float working precision):
  // five launches per basis vector and no host round trip until selection.
  void blur_dev(const Level<T>& L, bool tr, const Acc* x, Acc* y, const double* nrm2, Acc* xcopy) {
    if (blur_direct(L, tr, x, y, 1.f, nrm2, xcopy)) return;
    BandOp<Acc> op = L.op(H.nterms);
    const int sm = smem_bytes(op);
    if (sm > 48 * 1024) require_smem_limit((const void*)k_blur<Acc, Acc>, sm);
    const int nt = L.ntiles_side();
    const int grid = std::min(nt * nt, ctx->nsm * 8);
    { count_launch(); k_blur<Acc, Acc><<<grid, dim3(32, TY), sm, st>>>(op, tr ? 1 : 0, x, y, Acc(1), nrm2, xcopy); }
    CK(cudaGetLastError());
  }

  // the chunk partials of nslot outputs in gpart2 -> their destinations
  template <class Map> void part_reduce(int nslot, int nch, const float2* part, const Map& map) {
    if (nslot <= 0) return;
    count_launch();
    k_part_reduce<Map><<<(nslot + 7) / 8, 256, 0, st>>>(nslot, nch, part, map);
  }

  // k_vchunk and its reduction: dots into out[r * ostride] (VCH_DOTS), the
  // norm into *outnorm (VCH_NORM)
  void vchunk(size_t n, int nrows, const float* V, const double* coef, int cstride, float* x, int mode, double* out,
              int ostride, double* outnorm, int nch, int E) {
    REQUIRE((size_t)(nrows + 1) * nch <= gpart2_cap, "Gram partial buffer too small");
    count_launch();
    k_vchunk<<<nch, VCH_THREADS, 0, st>>>(n, nrows, V, n, coef, cstride, x, mode, gpart2, E);
    const int r0 = (mode & VCH_DOTS) ? 0 : nrows;
    const int r1 = (mode & VCH_NORM) ? nrows + 1 : nrows;
    part_reduce(r1 - r0, nch, gpart2 + (size_t)r0 * nch, RedRows{r0, nrows, ostride, out, outnorm});
  }

  // k_gram_col and its reduction into G_A, G_D, g_A, g_D (t == null: D part only)
  void gram_col(int m, int nr, const float* vj, int jout, const float* V, const float* t, const T* wx, const T* wy,
                const float* atbf, const float* dtcf, int nch, int E) {
    REQUIRE((size_t)2 * (nr + 2) * nch <= gpart2_cap, "Gram partial buffer too small");
    count_launch();
    k_gram_col<T><<<nch, VCH_THREADS, 0, st>>>(m, nr, vj, jout, V, t, wx, wy, atbf, dtcf, gpart2, E);
    part_reduce(2 * (nr + 2), nch, gpart2, RedGramCol{nr, jout, gkmax, t != nullptr ? 1 : 0, gGA, gGD, ggA, ggD});
  }

  // G_D[i][j], i <= j < kk, of V_0..V_{kk-1} for the weights (wx, wy) (null:
  // unweighted): k_gram_dtd over ~2 blocks per SM, then k_gram_dtd_reduce
  void gram_dtd(int m, int kk, const float* V, const T* wx, const T* wy, int ld) {
    REQUIRE(kk >= 1 && kk <= SK_KMAX, "G_D kernel takes at most 165 basis vectors");
    const size_t n = (size_t)m * m;
    size_t ppb = (n + (size_t)2 * ctx->nsm - 1) / ((size_t)2 * ctx->nsm);
    ppb = std::max<size_t>((ppb + SK_PC - 1) / SK_PC * SK_PC, SK_PC);
    const size_t nblk = (n + ppb - 1) / ppb;
    REQUIRE(nblk <= gsk_blocks, "G_D partial buffer too small");
    count_launch();
    k_gram_dtd<T><<<(unsigned)nblk, SK_THREADS, 0, st>>>(m, kk, V, wx, wy, (int)ppb, gsk);
    const int nb = (kk + SK_TI - 1) / SK_TI;
    const int nslot = nb * (nb + 1) / 2 * SK_TI * SK_TI;
    count_launch();
    k_gram_dtd_reduce<<<(nslot + 31) / 32, 256, 0, st>>>((int)nblk, kk, gsk, gGD, ld);
    CK(cudaGetLastError());
  }

  double gcv_projected_fused(const Level<T>& L, const T* wx, const T* wy, bool has_c, double s, double bnorm2,
                             double atb2, bool kc_hit) {
    const size_t n = L.n;
    const int m = L.m;
    const int ld = gkmax;
    GcvBufs<Acc>& C = *gcur;
    // chunk of E*256 elements per block, E chosen to give ~2 blocks per SM
    int E = VCH_E;
    while (E > 1 && (n + (size_t)E * VCH_THREADS - 1) / ((size_t)E * VCH_THREADS) < (size_t)2 * ctx->nsm) E >>= 1;
    const int nch = (int)((n + (size_t)E * VCH_THREADS - 1) / ((size_t)E * VCH_THREADS));
    float* V = reinterpret_cast<float*>(gV);
    float* t = reinterpret_cast<float*>(gt);
    const float* atbf = reinterpret_cast<const float*>(gatb);
    const float* dtcf = has_c ? reinterpret_cast<const float*>(gdtc) : nullptr;
    // the shift direction orth(D^T c) lives in the last slot of V and of the
    // Gram matrices, so it never overwrites a cached Krylov column
    const int kres = gkmax - 1;
    if (!kc_hit) {
      // start the basis: pending first direction t = A^T b with ||t||^2 = atb2
      CK(cudaMemcpyAsync(t, gatb, n * sizeof(float), cudaMemcpyDeviceToDevice, st));
      CK(cudaMemcpyAsync(C.gpend, &atb2, sizeof(double), cudaMemcpyHostToDevice, st));
      C.kc_b = (const void*)L.b;
      C.kc_epoch = epoch;
      C.kc_cols = 0;
      C.kc_bnorm2 = bnorm2;
      C.kc_atb2 = atb2;
    }
    const int cached = C.kc_cols;     // columns whose G_A, g_A are known; their G_D, g_D are stale
    const double dtc2 = has_c ? dot(n, gdtc, gdtc) : 0.0;
    const int kcap = (int)std::min<size_t>((size_t)std::min(go.proj_dim_max, kres - 2), n);
    // the doubling sequence k = proj_dim, 2 proj_dim, ... (<= kcap); every
    // selection of it runs in one launch and the rule is applied afterwards
    // (the result is the one the sequential loop returns)
    std::vector<int> seq;
    for (int k = std::min<int>(go.proj_dim, kcap);; k *= 2) {
      seq.push_back(k);
      if (2 * k > kcap || k >= (int)n) break;
    }
    const int ktop = seq.back();
    // new columns: v_j = t / ||t|| (written by the A pass), z = A v_j, t = A^T z
    while (C.kc_cols < ktop) {
      const int j = C.kc_cols;
      blur_dev(L, false, gt, gz, C.gpend, gV + (size_t)j * n);
      blur_dev(L, true, gz, gt, nullptr, nullptr);
      gram_col(m, j, V + (size_t)j * n, j, V, t, wx, wy, atbf, dtcf, nch, E);
      ++C.kc_cols;
      if (C.kc_cols < kcap) {
        // next direction: two classical Gram-Schmidt passes (the first reuses
        // the Gram column G_A[i][j] = V_i . t)
        vchunk(n, j + 1, V, gGA + j, ld, t, VCH_UPDATE | VCH_DOTS, gh, 1, nullptr, nch, E);
        vchunk(n, j + 1, V, gh, 1, t, VCH_UPDATE | VCH_NORM, nullptr, 0, C.gpend, nch, E);
      }
      CK(cudaGetLastError());
    }
    // G_D and g_D of the basis columns for the current weights and shift, in
    // one pass over V (the same arithmetic whether the columns were cached or
    // have just been built)
    gram_dtd(m, ktop, V, wx, wy, ld);
    if (dtcf) vchunk(n, ktop, V, nullptr, 0, const_cast<float*>(dtcf), VCH_DOTS, ggD, 1, nullptr, nch, E);
    else CK(cudaMemsetAsync(ggD, 0, (size_t)ktop * sizeof(double), st));
    CK(cudaGetLastError());
    // selections in groups of up to three per launch, the doubling rule
    // (stop at the first dimension whose gamma agrees with the previous one
    // to 0.1 %) applied in sequence order
    double gamma = 0.0, prev = -1.0;
    for (size_t g0 = 0; g0 < seq.size(); g0 += 3) {
      const int ng = (int)std::min<size_t>(3, seq.size() - g0);
      GcvSelectArgs args[3];
      size_t woff = 0;
      for (int bsel = 0; bsel < ng; ++bsel) {
        const int kdim = seq[g0 + bsel];
        const int kr = kres - bsel;       // slot of this selection's shift direction
        int kk = kdim, kshift = -1;
        if (has_c) {
          // shift direction orth(D^T c) against V_0..V_{kdim-1} (two Gram-Schmidt passes)
          float* vc = reinterpret_cast<float*>(gknext);
          CK(cudaMemcpyAsync(vc, gdtc, n * sizeof(float), cudaMemcpyDeviceToDevice, st));
          vchunk(n, kdim, V, nullptr, 0, vc, VCH_DOTS, gh, 1, nullptr, nch, E);
          vchunk(n, kdim, V, gh, 1, vc, VCH_UPDATE | VCH_DOTS, gh2, 1, nullptr, nch, E);
          vchunk(n, kdim, V, gh2, 1, vc, VCH_UPDATE | VCH_NORM, nullptr, 0, d_box + 22, nch, E);
          CK(cudaGetLastError());
          double nc2 = 0.0;
          CK(cudaMemcpyAsync(&nc2, d_box + 22, sizeof(double), cudaMemcpyDeviceToHost, st));
          CK(cudaStreamSynchronize(st));
          if (std::sqrt(nc2) > 1e-12 * std::sqrt(dtc2)) {
            float* vres = V + (size_t)kr * n;
            blur_dev(L, false, gknext, gz, d_box + 22, gV + (size_t)kr * n);
            blur_dev(L, true, gz, gy, nullptr, nullptr);
            gram_col(m, kdim, vres, kr, V, reinterpret_cast<float*>(gy), wx, wy, atbf, dtcf, nch, E);
            CK(cudaGetLastError());
            kk = kdim + 1;
            kshift = kr;
          }
        }
        GcvSelectArgs& a = args[bsel];
        a.kk = kk; a.ld = ld; a.GA = gGA; a.GD = gGD; a.gA = ggA; a.gD = ggD; a.kshift = kshift;
        a.bnorm2 = bnorm2; a.n = (double)n; a.s = s; a.rho = L.rho; a.npix = (int)n; a.exact = 0;
        a.lo = go.log10_gamma_lo; a.hi = go.log10_gamma_hi; a.tolx = go.refine_tol_log10;
        a.npts = go.grid_points; a.max_ext = 2; a.work = gwork + woff; a.out = d_box + 24 + 4 * bsel;
        woff += sel_work_doubles(kk);
      }
      REQUIRE(woff <= gwork_cap, "GCV selection workspace too small");
      const std::vector<double> gam = select_multi(args, ng);
      for (int i = 0; i < ng; ++i) {
        gamma = gam[i];
        if (prev > 0 && std::fabs(gamma - prev) <= 1e-3 * prev) return gamma;
        prev = gamma;
      }
    }
    return gamma;
  }

  // ---------------------------------------------------------------- outer step
  // x_new = x_old + delta, auxiliaries from L x_new; returns RC.
  double outer_update(Level<T>& L, int solver, const X* x_old, X* x_new) {
    const size_t n = L.n;
    const int g = grid_for(n, ctx->nsm);
    { count_launch(); k_outer_update<T><<<g, 256, 0, st>>>(L.m, solver, o.lsqr_warm_start, x_old, L.dlt, x_new, L.a0x, L.a0y,
                                         L.a1x, L.a1y, o.eps_irls, o.eps_mm, o.tau_sb, d_part, d_cnt + 4, d_box); }
    CK(cudaGetLastError());
    double h[2];
    CK(cudaMemcpyAsync(h, d_box, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    return h[1] == 0.0 ? INFINITY : std::sqrt(h[0]) / std::sqrt(h[1]);
  }

  // one level of Alg. 4 (Alg. 1/2/3 inside); x in L.xa on entry and exit
  void level_solve(Level<T>& L, int solver, double tol, bool twopass, double* mu, int* iters, int* inner) {
    X* x = L.xa;
    X* xn = L.xb;
    double gamma = 0.0;
    int k = 0, tot_inner = 0;
    for (k = 0; k < o.kmax; ++k) {
      if (solver == DB_IRLS) {
        if (!twopass) gamma = gcv(L, solver, true, false);
        else if (k == 0) gamma = gcv(L, solver, false, false);
        else if (k == 3) gamma = gcv(L, solver, true, false);
      } else if (k < go.gcv_estimates) {
        gamma = gcv(L, solver, false, true);
      }
      const int its = lsqr(L, solver, gamma, o.lsqr_warm_start ? x : nullptr);
      tot_inner += its;
      ctx->stats.outer_iterations++;
      const double rc = outer_update(L, solver, x, xn);
      std::swap(x, xn);
      if (rc < tol) { ++k; break; }
    }
    if (k > o.kmax) k = o.kmax;
    if (x != L.xa) CK(cudaMemcpyAsync(L.xa, x, L.n * sizeof(X), cudaMemcpyDeviceToDevice, st));
    *mu = gamma;
    *iters = k;
    *inner = tot_inner;
  }

  // Initial iterate and auxiliaries of level i (Alg. 4 / Sec. 4.1): the
  // coarsest level starts as Approach I; a finer level from the coarser
  // level's solution (Approach X) or auxiliary quantities (Approach D).
  void init_level(int i, db_solver solver, db_wavelet wv, db_transfer tr) {
    const Filter f = make_filter(wv);
    Level<T>& L = H.lv[i];
    const int g = grid_for(L.n, ctx->nsm);
    if (i == H.levels - 1) {
      { count_launch(); k_fill<X><<<g, 256, 0, st>>>(L.n, L.xa, 0.0); }
      { count_launch(); k_aux_init<T><<<g, 256, 0, st>>>(L.m, solver, AUX_APPROACH_I, L.xa, L.a0x, L.a0y, L.a1x,
            L.a1y, o.eps_irls, o.eps_mm, o.tau_sb); }
    } else {
      const Level<T>& C = H.lv[i + 1];
      if (tr == DB_APPROACH_X) {
        { count_launch(); k_prolong<X><<<g, 256, 0, st>>>(C.m, f, C.xa, L.xa, 0, 0); }
        { count_launch(); k_aux_init<T><<<g, 256, 0, st>>>(L.m, solver, AUX_FROM_X, L.xa, L.a0x, L.a0y, L.a1x,
              L.a1y, o.eps_irls, o.eps_mm, o.tau_sb); }
      } else {
        { count_launch(); k_fill<X><<<g, 256, 0, st>>>(L.n, L.xa, 0.0); }
        { count_launch(); k_prolong<T><<<g, 256, 0, st>>>(C.m, f, C.a0x, L.a0x, 1, 0); }
        { count_launch(); k_prolong<T><<<g, 256, 0, st>>>(C.m, f, C.a0y, L.a0y, 0, 1); }
        if (solver == DB_SB) {
          { count_launch(); k_prolong<T><<<g, 256, 0, st>>>(C.m, f, C.a1x, L.a1x, 1, 0); }
          { count_launch(); k_prolong<T><<<g, 256, 0, st>>>(C.m, f, C.a1y, L.a1y, 0, 1); }
        }
      }
    }
    CK(cudaGetLastError());
  }

  void vcycle(db_solver solver, db_wavelet wv, db_transfer tr, double* mu, int* iters, int* inner) {
    const int levels = H.levels;
    for (int i = levels - 1; i >= 0; --i) {
      init_level(i, solver, wv, tr);
      const double tol = i > 0 ? o.tol_coarse : o.tol_fine;
      const bool twopass = (solver == DB_IRLS && levels >= 3 && i == 0);
      level_solve(H.lv[i], solver, tol, twopass, &mu[i], &iters[i], &inner[i]);
    }
  }

  // x_new = x_old + delta and auxiliaries, without waiting; the two RC norms
  // land in out[0..1].
  void outer_update_async(Level<T>& L, int solver, const X* x_old, X* x_new, double* out) {
    const int g = grid_for(L.n, ctx->nsm);
    { count_launch(); k_outer_update<T><<<g, 256, 0, st>>>(L.m, solver, o.lsqr_warm_start, x_old, L.dlt, x_new,
          L.a0x, L.a0y, L.a1x, L.a1y, o.eps_irls, o.eps_mm, o.tau_sb, d_part, d_cnt + 4, out); }
    CK(cudaGetLastError());
  }
};

// ============================================================================
// batched solves: many V-cycles advanced together (one outer iteration of
// every unfinished problem per scheduler step)
// ============================================================================
// Persistent worker threads of the batched solver's GCV evaluations: run(f,
// n) calls f(0) .. f(n-1) on n workers and returns when all have returned.
// Starting threads once per solve (not once per scheduler step) keeps the
// step's fixed cost to a wake-up and a join.
struct WorkerPool {
  std::vector<std::thread> th;
  std::mutex mu;
  std::condition_variable cv, done;
  std::function<void(int)> job;
  unsigned gen = 0;
  int active = 0, pending = 0;
  bool stop = false;

  void start(int n, int device) {
    for (int w = 0; w < n; ++w)
      th.emplace_back([this, w, device]() {
        cudaSetDevice(device);
        unsigned seen = 0;
        for (;;) {
          std::function<void(int)> f;
          {
            std::unique_lock<std::mutex> lk(mu);
            cv.wait(lk, [&]() { return stop || gen != seen; });
            if (stop) return;
            seen = gen;
            if (w >= active) continue;
            f = job;
          }
          f(w);
          {
            std::lock_guard<std::mutex> lk(mu);
            if (--pending == 0) done.notify_all();
          }
        }
      });
  }
  void run(const std::function<void(int)>& f, int n) {
    std::unique_lock<std::mutex> lk(mu);
    job = f;
    active = n;
    pending = n;
    ++gen;
    cv.notify_all();
    done.wait(lk, [&]() { return pending == 0; });
  }
  ~WorkerPool() {
    {
      std::lock_guard<std::mutex> lk(mu);
      stop = true;
    }
    cv.notify_all();
    for (auto& t : th) t.join();
  }
};

template <typename T>
struct BatchSolver {
  using Acc = typename Traits<T>::Acc;
  using X = typename Traits<T>::X;
  struct Prob {
    std::unique_ptr<Engine<T>> E;
    db_solver solver;
    db_wavelet wv;
    db_transfer tr;
    int levels = 0, level = 0, k = 0, inner = 0;
    double gamma = 0.0;
    bool done = false;
    X* x = nullptr;
    X* xn = nullptr;
    std::vector<double> mu;
    std::vector<int> iters, inners;
    // GCV workspace of this problem: its Krylov basis stays cached across
    // the outer iterations of a level, as in a single solve
    GcvBufs<Acc> gb;
  };
  db_context* ctx;
  cudaStream_t st;
  db_opts o;
  db_gcv_opts go;
  std::vector<Prob> P;
  std::vector<cudaStream_t> wst;
  std::unique_ptr<WorkerPool> pool;   // GCV workers (one per worker stream)
  LsqrProb<T, Acc>* d_probs = nullptr;
  LsqrState* d_states = nullptr;
  LsqrCoef<Acc>* d_coefs = nullptr;
  int* d_tile_prob = nullptr;
  double* d_part = nullptr;
  GridBarrier* d_gb = nullptr;
  double* d_rc = nullptr;
  size_t max_tiles = 0;

  BatchSolver(db_context* c, cudaStream_t s) : ctx(c), st(s) {}
  ~BatchSolver() {
    pool.reset();
    P.clear();
    for (auto w : wst) cudaStreamDestroy(w);
  }

  static int workers_for(int count) { return std::max(1, std::min(count, 8)); }

  // device bytes of one problem: its levels and its GCV workspace
  static size_t problem_bytes(int m, int levels, int psf_size, const db_gcv_opts& g, int nsm) {
    return Engine<T>::footprint_levels(m, levels, psf_size) + (4ull << 20) +
           GcvBufs<Acc>::bytes((size_t)m * m, Engine<T>::gram_dim(g), g.exact_max_pixels, nsm);
  }

  static size_t footprint(int count, const db_request* r, const db_gcv_opts& g, int nsm) {
    size_t tot = 0, tiles = 0;
    for (int i = 0; i < count; ++i) {
      tot += problem_bytes(r[i].m, r[i].levels, r[i].psf_size, g, nsm);
      tiles += (size_t)((r[i].m + TM - 1) / TM) * ((r[i].m + TM - 1) / TM);
    }
    tot += (size_t)count * (sizeof(LsqrProb<T, Acc>) + sizeof(LsqrState) + sizeof(LsqrCoef<Acc>) + 4 * 256 + 64);
    tot += tiles * (6 * sizeof(double) + sizeof(int)) + (16ull << 20);
    return tot;
  }

  // Shared buffers: batched-LSQR tables for up to max_probs problems and
  // max_tiles tiles, and the worker streams of the GCV evaluations.
  void alloc_shared(Arena& A, int max_probs, size_t tiles, int nworkers) {
    max_tiles = tiles;
    wst.resize(nworkers);
    for (int w = 0; w < nworkers; ++w) CK(cudaStreamCreateWithFlags(&wst[w], cudaStreamNonBlocking));
    pool.reset(new WorkerPool());
    pool->start(nworkers, ctx->device);
    d_probs = A.take<LsqrProb<T, Acc>>(max_probs);
    d_states = A.take<LsqrState>(max_probs);
    d_coefs = A.take<LsqrCoef<Acc>>(max_probs);
    d_tile_prob = A.take<int>(max_tiles + 1);
    d_part = A.take<double>(6 * max_tiles + 6);   // LSQR tile partials, two phase buffers
    d_gb = A.take<GridBarrier>(1);
    d_rc = A.take<double>(2 * (size_t)max_probs);
    P.resize(max_probs);
    for (auto& q : P) q.done = true;
  }

  // Put a problem into slot i and start its coarsest level.
  void add_problem(int i, const db_request& r, const double* b_dev, const double* psf_dev, Arena* own) {
    Prob& q = P[i];
    q.E.reset(new Engine<T>(ctx, st));
    q.E->o = o;
    q.E->go = go;
    q.E->arena = own;
    q.solver = r.solver;
    q.wv = r.wavelet;
    q.levels = r.levels;
    q.tr = q.levels == 1 ? DB_APPROACH_I : r.transfer;
    q.E->build(psf_dev, r.psf_size, r.m, q.levels, q.wv, b_dev, true, false);
    q.gb.alloc(own ? *own : ctx->arena, (size_t)r.m * r.m, Engine<T>::gram_dim(go), go.exact_max_pixels, ctx->nsm);
    q.mu.assign(q.levels, 0.0);
    q.iters.assign(q.levels, 0);
    q.inners.assign(q.levels, 0);
    q.level = q.levels - 1;
    q.done = false;
    start_level(q);
  }

  void setup(int count, const db_request* reqs, const double* const* b_dev, const double* const* psf_dev) {
    size_t tiles = 0;
    for (int i = 0; i < count; ++i) tiles += (size_t)((reqs[i].m + TM - 1) / TM) * ((reqs[i].m + TM - 1) / TM);
    alloc_shared(ctx->arena, count, tiles, workers_for(count));
    for (int i = 0; i < count; ++i) add_problem(i, reqs[i], b_dev[i], psf_dev[i], nullptr);
    CK(cudaStreamSynchronize(st));
  }

  void start_level(Prob& q) {
    q.E->st = st;
    q.E->init_level(q.level, q.solver, q.wv, q.tr);
    Level<T>& L = q.E->H.lv[q.level];
    q.x = L.xa;
    q.xn = L.xb;
    q.k = 0;
    q.inner = 0;
  }

  // 0: no GCV this iteration; otherwise 1 + (weighted ? 1 : 0) + (shifted ? 2 : 0)
  int gcv_kind(const Prob& q) const {
    if (q.solver == DB_IRLS) {
      const bool twopass = q.levels >= 3 && q.level == 0;
      if (!twopass) return 1 + 1;
      if (q.k == 0) return 1;
      if (q.k == 3) return 1 + 1;
      return 0;
    }
    return q.k < go.gcv_estimates ? 1 + 2 : 0;
  }

  void run_gcvs(const std::vector<int>& need) {
    if (need.empty()) return;
    // the GCV evaluations run on the worker streams and read what the main
    // stream wrote last: a new level's right-hand side and auxiliaries
    // (start_level), a newly admitted problem's hierarchy (add_problem)
    CK(cudaStreamSynchronize(st));
    const int nw = std::min((int)wst.size(), (int)need.size());
    std::vector<DbError> errs(nw);
    std::vector<int> failed(nw, 0);
    auto work = [&](int w) {
      CountScope cs(ctx);
      try {
        // every problem has its own GCV buffers (and cached Krylov basis),
        // so the evaluations are dealt to the workers in turn
        for (size_t j = 0; j < need.size(); ++j) {
          if ((int)(j % nw) != w) continue;
          Prob& q = P[need[j]];
          const int kind = gcv_kind(q);
          q.E->adopt(q.gb);
          q.E->st = wst[w];
          // the level's x and auxiliaries were written on the main stream,
          // which the scheduler has synchronised before this point
          q.gamma = q.E->gcv(q.E->H.lv[q.level], q.solver, (kind - 1) & 1, ((kind - 1) & 2) != 0);
          q.E->st = st;
        }
      } catch (DbError& e) {
        errs[w] = e;
        failed[w] = 1;
      }
    };
    // a single evaluation runs on the calling thread
    if (nw == 1) work(0);
    else pool->run(work, nw);
    for (int w = 0; w < nw; ++w)
      if (failed[w]) throw errs[w];
  }

  void lsqr_batch(const std::vector<int>& act, std::vector<int>& its) {
    std::vector<LsqrProb<T, Acc>> hp(act.size());
    std::vector<int> tp;
    int sm = 0;
    for (size_t j = 0; j < act.size(); ++j) {
      Prob& q = P[act[j]];
      Engine<T>& E = *q.E;
      Level<T>& L = E.H.lv[q.level];
      LsqrProb<T, Acc>& X = hp[j];
      X.op = L.op(E.H.nterms);
      X.m = L.m;
      X.solver = q.solver;
      X.gamma = q.gamma;
      X.sg = (Acc)std::sqrt(q.gamma);
      X.b = L.b;
      X.x0 = o.lsqr_warm_start ? q.x : nullptr;
      X.a0x = L.a0x; X.a0y = L.a0y; X.a1x = L.a1x; X.a1y = L.a1y;
      X.uA = L.uA; X.uLx = L.uLx; X.uLy = L.uLy; X.v = L.v; X.w = L.wv; X.dlt = L.dlt;
      X.nt = L.ntiles_side();
      X.ntiles = X.nt * X.nt;
      X.tile_begin = (int)tp.size();
      Engine<T>::set_direct(X, L, X.x0);
      if (X.op.toep) ctx->stats.lsqr_direct_solves++;
      for (int t = 0; t < X.ntiles; ++t) tp.push_back((int)j);
      sm = std::max(sm, E.smem_bytes(X.op));
    }
    const int np = (int)act.size();
    CK(cudaMemcpyAsync(d_probs, hp.data(), sizeof(LsqrProb<T, Acc>) * np, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(d_tile_prob, tp.data(), sizeof(int) * tp.size(), cudaMemcpyHostToDevice, st));
    LsqrCtl c;
    c.atol = o.lsqr_atol; c.btol = o.lsqr_btol; c.conlim = o.lsqr_conlim; c.maxit = o.lsqr_maxit;
    c.nprob = np; c.ntiles = (int)tp.size();
    c.tile_prob = d_tile_prob; c.part = d_part; c.cnt = nullptr; c.st = d_states; c.gb = d_gb; c.coef = d_coefs;
    c.limit_ns = (unsigned long long)o.barrier_timeout_us * 1000ull;
    std::vector<BandOp<Acc>> ops(np);
    for (int j = 0; j < np; ++j) ops[j] = hp[j].op;
    auto reset = [&]() {
      CK(cudaMemsetAsync(d_states, 0, sizeof(LsqrState) * np, st));
      CK(cudaMemsetAsync(d_coefs, 0, sizeof(LsqrCoef<Acc>) * np, st));
      CK(cudaMemsetAsync(d_gb, 0, sizeof(GridBarrier), st));
    };
    const float lsqr_ms = lsqr_run<T, Acc>(ctx, st, d_probs, c, (int)tp.size(), sm, ops.data(), np, d_gb, reset);
    std::vector<LsqrState> S(np);
    GridBarrier gbh;
    CK(cudaMemcpyAsync(S.data(), d_states, sizeof(LsqrState) * np, cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(&gbh, d_gb, sizeof(gbh), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (gbh.error) throw DbError{DB_ETIMEOUT, "LSQR grid barrier timed out"};
    its.resize(np);
    ctx->stats.lsqr_launches++;
    for (int j = 0; j < np; ++j) {
      its[j] = S[j].its;
      const Prob& q = P[act[j]];
      const double pix = (double)(S[j].its + 1) * (double)q.E->H.lv[q.level].n;
      if (q.solver == DB_IRLS) ctx->stats.lsqr_pixel_iters_irls += pix;
      else ctx->stats.lsqr_pixel_iters_other += pix;
    }
    if (ctx->profiling) ctx->stats.lsqr_ms += lsqr_ms;
  }

  // One scheduler step: one outer iteration of every unfinished problem.
  // Returns the slots whose finest level completed in this step.
  std::vector<int> step() {
    std::vector<int> act, need, finished;
    for (int i = 0; i < (int)P.size(); ++i)
      if (!P[i].done) {
        act.push_back(i);
        if (gcv_kind(P[i])) need.push_back(i);
      }
    if (act.empty()) return finished;
    run_gcvs(need);
    std::vector<int> its;
    lsqr_batch(act, its);
    for (size_t j = 0; j < act.size(); ++j) {
      Prob& q = P[act[j]];
      q.E->outer_update_async(q.E->H.lv[q.level], q.solver, q.x, q.xn, d_rc + 2 * act[j]);
    }
    std::vector<double> rc(2 * P.size());
    CK(cudaMemcpyAsync(rc.data(), d_rc, sizeof(double) * rc.size(), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    ctx->stats.outer_iterations += act.size();
    for (size_t j = 0; j < act.size(); ++j) {
      Prob& q = P[act[j]];
      const int i = act[j];
      q.inner += its[j];
      std::swap(q.x, q.xn);
      ++q.k;
      const double r = rc[2 * i + 1] == 0.0 ? INFINITY : std::sqrt(rc[2 * i]) / std::sqrt(rc[2 * i + 1]);
      const double tol = q.level > 0 ? o.tol_coarse : o.tol_fine;
      if (r < tol || q.k >= o.kmax) {
        Level<T>& L = q.E->H.lv[q.level];
        if (q.x != L.xa) CK(cudaMemcpyAsync(L.xa, q.x, L.n * sizeof(X), cudaMemcpyDeviceToDevice, st));
        q.mu[q.level] = q.gamma;
        q.iters[q.level] = q.k;
        q.inners[q.level] = q.inner;
        if (q.level == 0) {
          q.E->check_blur_err();
          q.done = true;
          finished.push_back(i);
        } else {
          --q.level;
          start_level(q);
        }
      }
    }
    return finished;
  }

  void run() {
    for (;;) {
      bool any = false;
      for (auto& q : P) any |= !q.done;
      if (!any) break;
      step();
    }
  }
};

// ============================================================================
// C-ABI
// ============================================================================
extern "C" void db_default_opts(db_opts* o, db_gcv_opts* g) {
  if (o) {
    o->tol_fine = 1e-3; o->tol_coarse = 1e-6; o->kmax = 50;
    o->eps_irls = 0.03; o->eps_mm = 0.03; o->tau_sb = 0.005;
    o->lsqr_atol = 1e-6; o->lsqr_btol = 1e-6; o->lsqr_conlim = 1e8; o->lsqr_maxit = 100;
    o->lsqr_warm_start = 1; o->precision = DB_PREC_FP32;
    o->barrier_timeout_us = 2000000;
    o->fine_direct = 1;
  }
  if (g) {
    g->grid_points = 50; g->log10_gamma_lo = -10.0; g->log10_gamma_hi = 2.0;
    g->refine_tol_log10 = 1e-5; g->gcv_estimates = 3; g->proj_dim = 40; g->proj_dim_max = 160;
    g->gamma_fixed = 0.0; g->exact_max_pixels = 256;
  }
}

extern "C" const char* db_last_error(db_context* ctx) { return ctx ? ctx->err.c_str() : g_last_error.c_str(); }

extern "C" db_status db_context_create(db_context** out, int device, size_t budget) {
  if (!out) return DB_EINVAL;
  try {
    int ndev = 0;
    CK(cudaGetDeviceCount(&ndev));
    REQUIRE(device >= 0 && device < ndev, "no such CUDA device");
    CK(cudaSetDevice(device));
    db_context* c = new db_context();
    c->device = device;
    c->arena.budget = budget;
    CK(cudaDeviceGetAttribute(&c->nsm, cudaDevAttrMultiProcessorCount, device));
    *out = c;
    return DB_OK;
  } catch (DbError& e) {
    g_last_error = e.msg;
    return e.st;
  }
}

extern "C" db_status db_set_profiling(db_context* c, int on) {
  if (!c) return DB_EINVAL;
  try {
    CK(cudaSetDevice(c->device));
    if (on && !c->ev0) {
      CK(cudaEventCreate(&c->ev0));
      CK(cudaEventCreate(&c->ev1));
    }
    c->profiling = on ? 1 : 0;
    return DB_OK;
  } catch (DbError& e) {
    c->err = e.msg;
    return e.st;
  }
}

extern "C" db_status db_set_autotune(db_context* c, int on) {
  if (!c) return DB_EINVAL;
  c->autotune = on ? 1 : 0;
  return DB_OK;
}

extern "C" db_status db_get_stats(db_context* c, db_stats* out) {
  if (!c || !out) return DB_EINVAL;
  *out = c->stats;
  out->kernel_launches = c->n_launches.load();
  out->gcv_calls = c->n_gcv.load();
  out->gcv_ms = (double)c->gcv_ns.load() * 1e-6;
  out->blur_direct_launches = c->n_blur_direct.load();
  return DB_OK;
}

extern "C" db_status db_reset_stats(db_context* c) {
  if (!c) return DB_EINVAL;
  c->stats = db_stats{};
  c->n_launches = 0;
  c->n_gcv = 0;
  c->gcv_ns = 0;
  c->n_blur_direct = 0;
  return DB_OK;
}

extern "C" db_status db_context_destroy(db_context* c) {
  if (!c) return DB_EINVAL;
  cudaSetDevice(c->device);
  if (c->ev0) cudaEventDestroy(c->ev0);
  if (c->ev1) cudaEventDestroy(c->ev1);
  if (c->psf_fr) cudaFree(c->psf_fr);
  if (c->psf_fc) cudaFree(c->psf_fc);
  delete c;   // the arena frees its own block
  return DB_OK;
}

extern "C" size_t db_footprint_bytes(int m, int levels, int S, db_precision prec, const db_gcv_opts* gcv) {
  db_gcv_opts g;
  db_default_opts(nullptr, &g);
  if (gcv) g = *gcv;
  if (prec == DB_PREC_FP64) return Engine<double>::footprint(m, levels, S, g);
  if (prec == DB_PREC_BF16) return Engine<__nv_bfloat16>::footprint(m, levels, S, g);
  return Engine<float>::footprint(m, levels, S, g);
}

static void validate(int m, int S, int levels, db_wavelet wv) {
  REQUIRE(m >= 2 && (m & (m - 1)) == 0, "m must be a power of two");
  REQUIRE(S >= 1 && (S & 1) == 1 && S < m, "PSF size must be odd and smaller than m");
  REQUIRE(wv == DB_HAAR || wv == DB_DB4, "unknown wavelet");
  REQUIRE(levels >= 1 && levels <= 16, "levels out of range");
  const int kappa = wv == DB_HAAR ? 2 : 4;
  REQUIRE((m >> (levels - 1)) >= kappa && (m >> (levels - 1)) >= 2, "coarsest level smaller than the filter");
}

static void validate_opts(const db_opts& o, const db_gcv_opts& g) {
  REQUIRE(g.proj_dim >= 1 && g.proj_dim_max >= g.proj_dim && g.grid_points >= 3 && g.grid_points <= 64,
          "bad GCV options");
  REQUIRE(g.exact_max_pixels >= 0 && g.exact_max_pixels <= 1024, "exact_max_pixels out of range");
  REQUIRE(o.kmax >= 1 && o.lsqr_maxit >= 1, "bad iteration limits");
  REQUIRE(o.barrier_timeout_us >= 0, "barrier_timeout_us must be >= 0");
  REQUIRE(o.fine_direct == 0 || o.fine_direct == 1, "fine_direct must be 0 or 1");
}

template <typename T>
static void run_solve(db_context* ctx, cudaStream_t st, const double* b_dev, int m, const double* psf_dev, int S,
                      db_solver solver, db_wavelet wv, int levels, db_transfer tr, const db_gcv_opts& g,
                      const db_opts& o, double* x_dev, double* mu, int* iters, int* inner) {
  Engine<T> E(ctx, st);
  E.o = o;
  E.go = g;
  ctx->arena.ensure(Engine<T>::footprint(m, levels, S, g));
  ctx->arena.reset();
  E.build(psf_dev, S, m, levels, wv, b_dev, true);
  E.vcycle(solver, wv, levels == 1 ? DB_APPROACH_I : tr, mu, iters, inner);
  E.check_blur_err();
  { count_launch(); k_convert_out<typename Traits<T>::X><<<grid_for((size_t)m * m, ctx->nsm), 256, 0, st>>>((size_t)m * m, E.H.lv[0].xa, x_dev); }
  CK(cudaGetLastError());
}

extern "C" db_status deblur_solve(db_context* ctx, const double* b, int m, const double* psf, int S, db_solver solver,
                       db_wavelet wavelet, int levels, db_transfer transfer, const db_gcv_opts* gcv,
                       const db_opts* opts, double* x, double* mu_per_level, int* iters_per_level,
                       int* inner_iters_per_level, int on_device, db_stream stream) {
  if (!ctx) return DB_EINVAL;
  CountScope count_scope(ctx);
  cudaStream_t st = (cudaStream_t)stream;
  double *db_ = nullptr, *dpsf = nullptr, *dx = nullptr;   // staging copies of host arguments
  try {
    REQUIRE(b && psf && x && mu_per_level && iters_per_level, "null pointer argument");
    validate(m, S, levels, wavelet);
    REQUIRE(solver >= DB_IRLS && solver <= DB_SB, "unknown solver");
    REQUIRE(transfer >= DB_APPROACH_I && transfer <= DB_APPROACH_D, "unknown transfer strategy");
    db_opts o;
    db_gcv_opts g;
    db_default_opts(&o, &g);
    if (opts) o = *opts;
    if (gcv) g = *gcv;
    validate_opts(o, g);
    CK(cudaSetDevice(ctx->device));
    const size_t n = (size_t)m * m;
    if (!on_device) {
      CK(cudaMallocAsync((void**)&db_, n * sizeof(double), st));
      CK(cudaMallocAsync((void**)&dpsf, (size_t)S * S * sizeof(double), st));
      CK(cudaMallocAsync((void**)&dx, n * sizeof(double), st));
      CK(cudaMemcpyAsync(db_, b, n * sizeof(double), cudaMemcpyHostToDevice, st));
      CK(cudaMemcpyAsync(dpsf, psf, (size_t)S * S * sizeof(double), cudaMemcpyHostToDevice, st));
    } else {
      db_ = const_cast<double*>(b);
      dpsf = const_cast<double*>(psf);
      dx = x;
    }
    std::vector<double> mu(levels, 0.0);
    std::vector<int> it(levels, 0), inn(levels, 0);
    if (o.precision == DB_PREC_FP64)
      run_solve<double>(ctx, st, db_, m, dpsf, S, solver, wavelet, levels, transfer, g, o, dx, mu.data(), it.data(), inn.data());
    else if (o.precision == DB_PREC_BF16)
      run_solve<__nv_bfloat16>(ctx, st, db_, m, dpsf, S, solver, wavelet, levels, transfer, g, o, dx, mu.data(), it.data(), inn.data());
    else
      run_solve<float>(ctx, st, db_, m, dpsf, S, solver, wavelet, levels, transfer, g, o, dx, mu.data(), it.data(), inn.data());
    if (!on_device) {
      CK(cudaMemcpyAsync(x, dx, n * sizeof(double), cudaMemcpyDeviceToHost, st));
      CK(cudaFreeAsync(db_, st));
      CK(cudaFreeAsync(dpsf, st));
      CK(cudaFreeAsync(dx, st));
      db_ = dpsf = dx = nullptr;
    }
    CK(cudaStreamSynchronize(st));
    for (int i = 0; i < levels; ++i) {
      mu_per_level[i] = mu[i];
      iters_per_level[i] = it[i];
      if (inner_iters_per_level) inner_iters_per_level[i] = inn[i];
    }
    return DB_OK;
  } catch (DbError& e) {
    // nothing of this call may still run, or hold memory, when it returns
    cudaStreamSynchronize(st);
    if (!on_device) {
      if (db_) cudaFree(db_);
      if (dpsf) cudaFree(dpsf);
      if (dx) cudaFree(dx);
    }
    cudaGetLastError();
    ctx->err = e.msg;
    return e.st;
  }
}

template <typename T>
static void run_batch(db_context* ctx, cudaStream_t st, int count, const db_request* reqs, const db_gcv_opts& g,
                      const db_opts& o, const double* const* b_dev, const double* const* psf_dev,
                      double* const* x_dev) {
  BatchSolver<T> B(ctx, st);
  B.o = o;
  B.go = g;
  ctx->arena.ensure(BatchSolver<T>::footprint(count, reqs, g, ctx->nsm));
  ctx->arena.reset();
  B.setup(count, reqs, b_dev, psf_dev);
  B.run();
  for (int i = 0; i < count; ++i) {
    auto& q = B.P[i];
    const size_t n = (size_t)reqs[i].m * reqs[i].m;
    { count_launch(); k_convert_out<typename Traits<T>::X><<<grid_for(n, ctx->nsm), 256, 0, st>>>(n, q.E->H.lv[0].xa, x_dev[i]); }
    for (int l = 0; l < q.levels; ++l) {
      reqs[i].mu_per_level[l] = q.mu[l];
      reqs[i].iters_per_level[l] = q.iters[l];
      if (reqs[i].inner_iters_per_level) reqs[i].inner_iters_per_level[l] = q.inners[l];
    }
  }
  CK(cudaGetLastError());
}

extern "C" db_status deblur_solve_batch(db_context* ctx, int count, const db_request* reqs, const db_gcv_opts* gcv,
                                        const db_opts* opts, int on_device, db_stream stream) {
  if (!ctx) return DB_EINVAL;
  CountScope count_scope(ctx);
  std::vector<double*> tmp;
  cudaStream_t st = (cudaStream_t)stream;
  try {
    REQUIRE(count >= 1 && reqs, "empty batch");
    db_opts o;
    db_gcv_opts g;
    db_default_opts(&o, &g);
    if (opts) o = *opts;
    if (gcv) g = *gcv;
    validate_opts(o, g);
    for (int i = 0; i < count; ++i) {
      const db_request& r = reqs[i];
      REQUIRE(r.b && r.psf && r.x && r.mu_per_level && r.iters_per_level, "null pointer in a request");
      validate(r.m, r.psf_size, r.levels, r.wavelet);
      REQUIRE(r.solver >= DB_IRLS && r.solver <= DB_SB, "unknown solver");
      REQUIRE(r.transfer >= DB_APPROACH_I && r.transfer <= DB_APPROACH_D, "unknown transfer strategy");
    }
    CK(cudaSetDevice(ctx->device));
    std::vector<const double*> bd(count), pd(count);
    std::vector<double*> xd(count);
    for (int i = 0; i < count; ++i) {
      const db_request& r = reqs[i];
      const size_t n = (size_t)r.m * r.m, ps = (size_t)r.psf_size * r.psf_size;
      if (on_device) {
        bd[i] = r.b; pd[i] = r.psf; xd[i] = r.x;
      } else {
        double *b_, *p_, *x_;
        CK(cudaMallocAsync((void**)&b_, n * sizeof(double), st)); tmp.push_back(b_);
        CK(cudaMallocAsync((void**)&p_, ps * sizeof(double), st)); tmp.push_back(p_);
        CK(cudaMallocAsync((void**)&x_, n * sizeof(double), st)); tmp.push_back(x_);
        CK(cudaMemcpyAsync(b_, r.b, n * sizeof(double), cudaMemcpyHostToDevice, st));
        CK(cudaMemcpyAsync(p_, r.psf, ps * sizeof(double), cudaMemcpyHostToDevice, st));
        bd[i] = b_; pd[i] = p_; xd[i] = x_;
      }
    }
    if (o.precision == DB_PREC_FP64) run_batch<double>(ctx, st, count, reqs, g, o, bd.data(), pd.data(), xd.data());
    else if (o.precision == DB_PREC_BF16) run_batch<__nv_bfloat16>(ctx, st, count, reqs, g, o, bd.data(), pd.data(), xd.data());
    else run_batch<float>(ctx, st, count, reqs, g, o, bd.data(), pd.data(), xd.data());
    if (!on_device) {
      for (int i = 0; i < count; ++i)
        CK(cudaMemcpyAsync(reqs[i].x, xd[i], (size_t)reqs[i].m * reqs[i].m * sizeof(double), cudaMemcpyDeviceToHost, st));
    }
    for (double* t : tmp) cudaFreeAsync(t, st);
    CK(cudaStreamSynchronize(st));
    return DB_OK;
  } catch (DbError& e) {
    for (double* t : tmp) cudaFreeAsync(t, st);
    cudaStreamSynchronize(st);
    ctx->err = e.msg;
    return e.st;
  }
}


// ============================================================================
// serving loop
// ============================================================================
struct ServerJob {
  uint64_t ticket = 0;
  db_request req{};
  std::vector<double> b, psf;
  Arena* arena = nullptr;            // the workspace of its slot while resident
  double* dev_b = nullptr;
  double* dev_psf = nullptr;
  double* dev_x = nullptr;
  size_t bytes = 0;
  int slot = -1;
  bool done = false;
  bool cancel = false;               // withdrawn while resident: retired at the next step boundary
  db_status status = DB_OK;
  std::chrono::steady_clock::time_point t_submit, t_done;
};

struct db_server {
  db_context* ctx = nullptr;
  db_server_opts opts{};
  cudaStream_t st = nullptr;
  std::thread th;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  bool stopping = false;
  uint64_t next_ticket = 1;
  std::deque<ServerJob*> queue;
  std::map<uint64_t, std::unique_ptr<ServerJob>> jobs;
  Arena shared;                      // batched-LSQR tables and GCV workspaces
  std::unique_ptr<BatchSolver<float>> B;
  std::vector<ServerJob*> slots;
  std::vector<std::unique_ptr<Arena>> slot_arena;   // per-slot workspace, reused by successive requests
  size_t bytes_in_use = 0;
  std::string fatal;

  size_t job_bytes(const db_request& r) const {
    return BatchSolver<float>::problem_bytes(r.m, r.levels, r.psf_size, opts.gcv, ctx->nsm);
  }

  void loop() {
    CountScope cs(ctx);
    cudaSetDevice(ctx->device);
    for (;;) {
      // admission at a step boundary
      {
        std::unique_lock<std::mutex> lk(mu);
        // resident requests withdrawn by db_server_cancel leave first
        for (int i = 0; i < (int)slots.size(); ++i) {
          ServerJob* j = slots[i];
          if (!j || !j->cancel) continue;
          B->P[i].done = true;
          B->P[i].E.reset();
          j->arena = nullptr;
          bytes_in_use -= j->bytes;
          slots[i] = nullptr;
          j->status = DB_ECANCELLED;
          j->done = true;
          j->t_done = std::chrono::steady_clock::now();
          cv_done.notify_all();
        }
        bool any_resident = false;
        for (auto* j : slots) any_resident |= (j != nullptr);
        if (!any_resident && queue.empty()) {
          if (stopping) return;
          cv_work.wait(lk, [&] { return stopping || !queue.empty(); });
          if (stopping && queue.empty()) return;
        }
        while (!queue.empty()) {
          ServerJob* j = queue.front();
          int free_slot = -1;
          for (int i = 0; i < (int)slots.size(); ++i)
            if (!slots[i]) { free_slot = i; break; }
          if (free_slot < 0) break;
          if (opts.hbm_budget_bytes && bytes_in_use + j->bytes > opts.hbm_budget_bytes && bytes_in_use > 0) break;
          queue.pop_front();
          lk.unlock();
          try {
            const size_t n = (size_t)j->req.m * j->req.m, ps = (size_t)j->req.psf_size * j->req.psf_size;
            // the slot's workspace is kept between requests and grows only
            // when a larger request arrives (cudaFree would stall the device)
            Arena& sa = *slot_arena[free_slot];
            sa.ensure(j->bytes + 3 * n * sizeof(double) + ps * sizeof(double) + 4096);
            sa.reset();
            j->arena = &sa;
            j->dev_b = j->arena->take<double>(n);
            j->dev_psf = j->arena->take<double>(ps);
            j->dev_x = j->arena->take<double>(n);
            CK(cudaMemcpyAsync(j->dev_b, j->b.data(), n * sizeof(double), cudaMemcpyHostToDevice, st));
            CK(cudaMemcpyAsync(j->dev_psf, j->psf.data(), ps * sizeof(double), cudaMemcpyHostToDevice, st));
            B->add_problem(free_slot, j->req, j->dev_b, j->dev_psf, j->arena);
            lk.lock();
            slots[free_slot] = j;
            j->slot = free_slot;
            bytes_in_use += j->bytes;
          } catch (DbError& e) {
            lk.lock();
            j->status = e.st;
            j->done = true;
            j->t_done = std::chrono::steady_clock::now();
            j->arena = nullptr;
            cv_done.notify_all();
          }
        }
      }
      // one scheduler step over the resident solves
      std::vector<int> fin;
      try {
        fin = B->step();
      } catch (DbError& e) {
        std::lock_guard<std::mutex> lk(mu);
        fatal = e.msg;
        for (int i = 0; i < (int)slots.size(); ++i)
          if (slots[i]) {
            ServerJob* j = slots[i];
            j->status = e.st;
            j->done = true;
            j->t_done = std::chrono::steady_clock::now();
            B->P[i].done = true;
            B->P[i].E.reset();
            j->arena = nullptr;
            slots[i] = nullptr;
          }
        bytes_in_use = 0;
        cv_done.notify_all();
        continue;
      }
      for (int i : fin) {
        ServerJob* j = slots[i];
        auto& q = B->P[i];
        const size_t n = (size_t)j->req.m * j->req.m;
        try {
          { count_launch(); k_convert_out<float><<<grid_for(n, ctx->nsm), 256, 0, st>>>(n, q.E->H.lv[0].xa, j->dev_x); }
          CK(cudaMemcpyAsync(j->req.x, j->dev_x, n * sizeof(double), cudaMemcpyDeviceToHost, st));
          CK(cudaStreamSynchronize(st));
          for (int l = 0; l < q.levels; ++l) {
            j->req.mu_per_level[l] = q.mu[l];
            j->req.iters_per_level[l] = q.iters[l];
            if (j->req.inner_iters_per_level) j->req.inner_iters_per_level[l] = q.inners[l];
          }
        } catch (DbError& e) {
          j->status = e.st;
        }
        q.E.reset();
        std::lock_guard<std::mutex> lk(mu);
        j->arena = nullptr;
        bytes_in_use -= j->bytes;
        slots[i] = nullptr;
        j->done = true;
        j->t_done = std::chrono::steady_clock::now();
        cv_done.notify_all();
      }
    }
  }
};

extern "C" db_status db_server_create(db_context* ctx, const db_server_opts* o, db_server** out) {
  if (!ctx || !o || !out) return DB_EINVAL;
  CountScope count_scope(ctx);
  try {
    REQUIRE(o->max_resident >= 1 && o->max_resident <= 256, "max_resident out of range");
    REQUIRE(o->max_m >= 8 && (o->max_m & (o->max_m - 1)) == 0, "max_m must be a power of two");
    validate_opts(o->opts, o->gcv);
    CK(cudaSetDevice(ctx->device));
    std::unique_ptr<db_server> s(new db_server());
    s->ctx = ctx;
    s->opts = *o;
    s->opts.opts.precision = DB_PREC_FP32;
    CK(cudaStreamCreateWithFlags(&s->st, cudaStreamNonBlocking));
    s->B.reset(new BatchSolver<float>(ctx, s->st));
    s->B->o = s->opts.opts;
    s->B->go = s->opts.gcv;
    const size_t tiles = (size_t)o->max_resident * ((o->max_m + TM - 1) / TM) * ((o->max_m + TM - 1) / TM);
    const int nw = BatchSolver<float>::workers_for(o->max_resident);
    s->shared.ensure(tiles * 40 + (size_t)o->max_resident * 4096 + (16ull << 20));
    s->B->alloc_shared(s->shared, o->max_resident, tiles, nw);
    s->slots.assign(o->max_resident, nullptr);
    for (int i = 0; i < o->max_resident; ++i) s->slot_arena.emplace_back(new Arena());
    if (o->hbm_budget_bytes) for (auto& a : s->slot_arena) a->budget = o->hbm_budget_bytes;
    db_server* raw = s.release();
    raw->th = std::thread([raw] { raw->loop(); });
    *out = raw;
    return DB_OK;
  } catch (DbError& e) {
    ctx->err = e.msg;
    return e.st;
  }
}

extern "C" db_status db_server_submit(db_server* s, const db_request* r, uint64_t* ticket) {
  if (!s || !r || !ticket) return DB_EINVAL;
  try {
    REQUIRE(r->b && r->psf && r->x && r->mu_per_level && r->iters_per_level, "null pointer in the request");
    validate(r->m, r->psf_size, r->levels, r->wavelet);
    REQUIRE(r->m <= s->opts.max_m, "image larger than the server's max_m");
    REQUIRE(r->solver >= DB_IRLS && r->solver <= DB_SB, "unknown solver");
    REQUIRE(r->transfer >= DB_APPROACH_I && r->transfer <= DB_APPROACH_D, "unknown transfer strategy");
    std::unique_ptr<ServerJob> j(new ServerJob());
    j->req = *r;
    j->b.assign(r->b, r->b + (size_t)r->m * r->m);
    j->psf.assign(r->psf, r->psf + (size_t)r->psf_size * r->psf_size);
    j->bytes = s->job_bytes(*r);
    j->t_submit = std::chrono::steady_clock::now();
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stopping) return DB_EBUSY;
    j->ticket = s->next_ticket++;
    *ticket = j->ticket;
    s->queue.push_back(j.get());
    s->jobs[j->ticket] = std::move(j);
    s->cv_work.notify_one();
    return DB_OK;
  } catch (DbError& e) {
    s->ctx->err = e.msg;
    return e.st;
  }
}

extern "C" db_status db_server_poll(db_server* s, uint64_t ticket, int timeout_us, double* latency_ms) {
  if (!s) return DB_EINVAL;
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->jobs.find(ticket);
  if (it == s->jobs.end()) return DB_EINVAL;
  ServerJob* j = it->second.get();
  auto ready = [&] { return j->done; };
  if (timeout_us < 0) s->cv_done.wait(lk, ready);
  else if (!s->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), ready)) return DB_ETIMEOUT;
  if (latency_ms) *latency_ms = std::chrono::duration<double, std::milli>(j->t_done - j->t_submit).count();
  if (j->status != DB_OK && !s->fatal.empty()) s->ctx->err = s->fatal;
  return j->status;
}

extern "C" db_status db_server_cancel(db_server* s, uint64_t ticket) {
  if (!s) return DB_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->jobs.find(ticket);
  if (it == s->jobs.end()) return DB_EINVAL;
  ServerJob* j = it->second.get();
  if (j->done) return DB_OK;                    // finished already: nothing to withdraw
  auto q = std::find(s->queue.begin(), s->queue.end(), j);
  if (q != s->queue.end()) {                    // not admitted yet: leaves the queue at once
    s->queue.erase(q);
    j->status = DB_ECANCELLED;
    j->done = true;
    j->t_done = std::chrono::steady_clock::now();
    s->cv_done.notify_all();
  } else {
    j->cancel = true;                           // resident: the scheduler retires it
  }
  return DB_OK;
}

extern "C" db_status db_server_destroy(db_server* s) {
  if (!s) return DB_EINVAL;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stopping = true;
    s->cv_work.notify_all();
  }
  if (s->th.joinable()) s->th.join();
  cudaSetDevice(s->ctx->device);
  s->B.reset();
  if (s->st) cudaStreamDestroy(s->st);
  delete s;   // frees the shared arena
  return DB_OK;
}

// ---- operator-level entry points ---------------------------------------------
template <typename T>
static void op_blur(db_context* ctx, cudaStream_t st, const double* psf_host, int S, int m, db_wavelet wv, int level,
                    int tr, const void* x, void* y) {
  Engine<T> E(ctx, st);
  db_default_opts(&E.o, &E.go);
  ctx->arena.ensure(Engine<T>::footprint(m, level + 1, S, E.go));
  ctx->arena.reset();
  double* dpsf = ctx->arena.take<double>((size_t)S * S);
  CK(cudaMemcpyAsync(dpsf, psf_host, (size_t)S * S * sizeof(double), cudaMemcpyHostToDevice, st));
  E.build(dpsf, S, m, level + 1, wv, nullptr, false);
  E.blur_T(E.H.lv[level], tr != 0, (const T*)x, (T*)y);
  E.check_blur_err();
}

extern "C" db_status db_apply_blur(db_context* ctx, const double* psf_host, int S, int m, db_wavelet wv, int level, int tr,
                        const void* x, void* y, db_precision prec, db_stream stream) {
  if (!ctx) return DB_EINVAL;
  CountScope count_scope(ctx);
  try {
    REQUIRE(psf_host && x && y, "null pointer argument");
    validate(m, S, level + 1, wv);
    CK(cudaSetDevice(ctx->device));
    cudaStream_t st = (cudaStream_t)stream;
    if (prec == DB_PREC_FP64) op_blur<double>(ctx, st, psf_host, S, m, wv, level, tr, x, y);
    else if (prec == DB_PREC_FP32) op_blur<float>(ctx, st, psf_host, S, m, wv, level, tr, x, y);
    else REQUIRE(false, "operator entry points take FP64 or FP32 buffers");
    CK(cudaStreamSynchronize(st));
    return DB_OK;
  } catch (DbError& e) {
    ctx->err = e.msg;
    return e.st;
  }
}

template <typename F>
static db_status simple_call(F&& f) {
  try {
    f();
    return DB_OK;
  } catch (DbError& e) {
    g_last_error = e.msg;
    return e.st;
  }
}

static int dev_sms() {
  int d = 0, n = 0;
  cudaGetDevice(&d);
  cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, d);
  return n > 0 ? n : 1;
}

// Sum of squares through the reduction of the LSQR norms: each thread
// accumulates the squares of its PIX elements of a 1024-element tile
// (Sums3), tile_partial combines the block, problem_partials adds the tile
// partials in tile order.
template <typename T>
__global__ void __launch_bounds__(256) k_sumsq_tiles(size_t n, const T* __restrict__ x, double* __restrict__ part) {
  using Acc = typename Traits<T>::Acc;
  __shared__ double scratch[3 * 32];
  Sums3<Acc> red;
  const size_t base = (size_t)blockIdx.x * (TM * TN);
#pragma unroll
  for (int j = 0; j < PIX; ++j) {
    const size_t i = base + threadIdx.x + (size_t)TM * pix_col(j);
    if (i < n) red.sq(0, to_acc(x[i]));
  }
  tile_partial(red, part + (size_t)blockIdx.x * 3, scratch);
}
template <typename Acc>
__global__ void k_sumsq_finish(int ntiles, const double* __restrict__ part, double* __restrict__ out) {
  double tot[3];
  problem_partials<Acc>(part, ntiles, tot);
  if (threadIdx.x == 0) *out = tot[0];
}

extern "C" db_status db_sumsq(const void* x, size_t n, db_precision prec, double* out, db_stream stream) {
  return simple_call([&] {
    REQUIRE(x && out && n >= 1, "bad arguments");
    REQUIRE(prec == DB_PREC_FP64 || prec == DB_PREC_FP32 || prec == DB_PREC_BF16, "unknown precision");
    cudaStream_t st = (cudaStream_t)stream;
    const size_t ntiles = (n + TM * TN - 1) / (TM * TN);
    REQUIRE(ntiles <= (size_t)INT32_MAX, "vector too long");
    double* d = nullptr;
    CK(cudaMallocAsync((void**)&d, (ntiles * 3 + 1) * sizeof(double), st));
    const dim3 blk(32, TY);
    if (prec == DB_PREC_FP64) {
      k_sumsq_tiles<double><<<(unsigned)ntiles, blk, 0, st>>>(n, (const double*)x, d);
      k_sumsq_finish<double><<<1, 32, 0, st>>>((int)ntiles, d, d + ntiles * 3);
    } else if (prec == DB_PREC_FP32) {
      k_sumsq_tiles<float><<<(unsigned)ntiles, blk, 0, st>>>(n, (const float*)x, d);
      k_sumsq_finish<float><<<1, 32, 0, st>>>((int)ntiles, d, d + ntiles * 3);
    } else {
      k_sumsq_tiles<__nv_bfloat16><<<(unsigned)ntiles, blk, 0, st>>>(n, (const __nv_bfloat16*)x, d);
      k_sumsq_finish<float><<<1, 32, 0, st>>>((int)ntiles, d, d + ntiles * 3);
    }
    count_launch();
    count_launch();
    const cudaError_t e = cudaGetLastError();
    CK(cudaMemcpyAsync(out, d + ntiles * 3, sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaFreeAsync(d, st));
    CK(cudaStreamSynchronize(st));
    CK(e);
  });
}

extern "C" db_status db_apply_L(int m, const void* x, void* q, db_precision prec, db_stream stream) {
  return simple_call([&] {
    REQUIRE(m >= 2 && x && q, "bad arguments");
    cudaStream_t st = (cudaStream_t)stream;
    size_t n = (size_t)m * m;
    int g = grid_for(n, dev_sms());
    if (prec == DB_PREC_FP64) { count_launch(); k_L<double><<<g, 256, 0, st>>>(m, (const double*)x, (double*)q, (double*)q + n); }
    else if (prec == DB_PREC_FP32) { count_launch(); k_L<float><<<g, 256, 0, st>>>(m, (const float*)x, (float*)q, (float*)q + n); }
    else REQUIRE(false, "FP64 or FP32 only");
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(st));
  });
}

extern "C" db_status db_apply_Lt(int m, const void* q, void* x, db_precision prec, db_stream stream) {
  return simple_call([&] {
    REQUIRE(m >= 2 && x && q, "bad arguments");
    cudaStream_t st = (cudaStream_t)stream;
    size_t n = (size_t)m * m;
    int g = grid_for(n, dev_sms());
    if (prec == DB_PREC_FP64) { count_launch(); k_Lt<double><<<g, 256, 0, st>>>(m, (const double*)q, (const double*)q + n, (double*)x); }
    else if (prec == DB_PREC_FP32) { count_launch(); k_Lt<float><<<g, 256, 0, st>>>(m, (const float*)q, (const float*)q + n, (float*)x); }
    else REQUIRE(false, "FP64 or FP32 only");
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(st));
  });
}

extern "C" db_status db_restrict(int m, db_wavelet wv, const void* x, void* y, db_precision prec, db_stream stream) {
  return simple_call([&] {
    REQUIRE(m >= 4 && (m & (m - 1)) == 0 && x && y, "bad arguments (m must be a power of two)");
    REQUIRE(wv == DB_HAAR || wv == DB_DB4, "unknown wavelet");
    REQUIRE(m >= make_filter(wv).kappa, "m smaller than the filter");
    cudaStream_t st = (cudaStream_t)stream;
    int g = grid_for((size_t)m * m / 4, dev_sms());
    if (prec == DB_PREC_FP64) { count_launch(); k_restrict<double><<<g, 256, 0, st>>>(m, make_filter(wv), (const double*)x, (double*)y); }
    else if (prec == DB_PREC_FP32) { count_launch(); k_restrict<float><<<g, 256, 0, st>>>(m, make_filter(wv), (const float*)x, (float*)y); }
    else REQUIRE(false, "FP64 or FP32 only");
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(st));
  });
}

extern "C" db_status db_prolong(int mc, db_wavelet wv, const void* y, void* x, db_precision prec, db_stream stream) {
  return simple_call([&] {
    REQUIRE(mc >= 1 && (mc & (mc - 1)) == 0 && x && y, "bad arguments (mc must be a power of two)");
    REQUIRE(wv == DB_HAAR || wv == DB_DB4, "unknown wavelet");
    REQUIRE(2 * mc >= make_filter(wv).kappa, "m smaller than the filter");
    cudaStream_t st = (cudaStream_t)stream;
    int g = grid_for((size_t)mc * mc * 4, dev_sms());
    if (prec == DB_PREC_FP64) { count_launch(); k_prolong<double><<<g, 256, 0, st>>>(mc, make_filter(wv), (const double*)y, (double*)x, 0, 0); }
    else if (prec == DB_PREC_FP32) { count_launch(); k_prolong<float><<<g, 256, 0, st>>>(mc, make_filter(wv), (const float*)y, (float*)x, 0, 0); }
    else REQUIRE(false, "FP64 or FP32 only");
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(st));
  });
}

extern "C" db_status db_aux_prolong(int mc, db_wavelet wv, const void* qc, void* qf, db_precision prec, db_stream stream) {
  return simple_call([&] {
    REQUIRE(mc >= 1 && (mc & (mc - 1)) == 0 && qc && qf, "bad arguments (mc must be a power of two)");
    REQUIRE(wv == DB_HAAR || wv == DB_DB4, "unknown wavelet");
    REQUIRE(2 * mc >= make_filter(wv).kappa, "m smaller than the filter");
    cudaStream_t st = (cudaStream_t)stream;
    const size_t nc = (size_t)mc * mc, nf = nc * 4;
    int g = grid_for(nf, dev_sms());
    Filter f = make_filter(wv);
    if (prec == DB_PREC_FP64) {
      { count_launch(); k_prolong<double><<<g, 256, 0, st>>>(mc, f, (const double*)qc, (double*)qf, 1, 0); }
      { count_launch(); k_prolong<double><<<g, 256, 0, st>>>(mc, f, (const double*)qc + nc, (double*)qf + nf, 0, 1); }
    } else if (prec == DB_PREC_FP32) {
      { count_launch(); k_prolong<float><<<g, 256, 0, st>>>(mc, f, (const float*)qc, (float*)qf, 1, 0); }
      { count_launch(); k_prolong<float><<<g, 256, 0, st>>>(mc, f, (const float*)qc + nc, (float*)qf + nf, 0, 1); }
    } else REQUIRE(false, "FP64 or FP32 only");
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(st));
  });
}

template <typename T>
static void op_lsqr(db_context* ctx, cudaStream_t st, const double* psf_host, int S, int m, db_solver solver,
                    double gamma, const void* b, const void* x0, const void* aux0, const void* aux1, void* x_out,
                    const db_opts& o, int* iters) {
  Engine<T> E(ctx, st);
  db_default_opts(nullptr, &E.go);
  E.o = o;
  ctx->arena.ensure(Engine<T>::footprint(m, 1, S, E.go));
  ctx->arena.reset();
  double* dpsf = ctx->arena.take<double>((size_t)S * S);
  CK(cudaMemcpyAsync(dpsf, psf_host, (size_t)S * S * sizeof(double), cudaMemcpyHostToDevice, st));
  E.build(dpsf, S, m, 1, DB_HAAR, nullptr, true);
  Level<T>& L = E.H.lv[0];
  const size_t n = L.n;
  CK(cudaMemcpyAsync(L.b, b, n * sizeof(T), cudaMemcpyDeviceToDevice, st));
  const T* a0 = (const T*)aux0;
  const T* a1 = (const T*)aux1;
  if (a0) {
    CK(cudaMemcpyAsync(L.a0x, a0, n * sizeof(T), cudaMemcpyDeviceToDevice, st));
    CK(cudaMemcpyAsync(L.a0y, a0 + n, n * sizeof(T), cudaMemcpyDeviceToDevice, st));
  } else {
    { count_launch(); k_fill<T><<<grid_for(n, ctx->nsm), 256, 0, st>>>(n, L.a0x, solver == DB_IRLS ? 1.0 : 0.0); }
    { count_launch(); k_fill<T><<<grid_for(n, ctx->nsm), 256, 0, st>>>(n, L.a0y, solver == DB_IRLS ? 1.0 : 0.0); }
  }
  if (a1) {
    CK(cudaMemcpyAsync(L.a1x, a1, n * sizeof(T), cudaMemcpyDeviceToDevice, st));
    CK(cudaMemcpyAsync(L.a1y, a1 + n, n * sizeof(T), cudaMemcpyDeviceToDevice, st));
  } else {
    { count_launch(); k_fill<T><<<grid_for(n, ctx->nsm), 256, 0, st>>>(n, L.a1x, 0.0); }
    { count_launch(); k_fill<T><<<grid_for(n, ctx->nsm), 256, 0, st>>>(n, L.a1y, 0.0); }
  }
  if (x0) CK(cudaMemcpyAsync(L.xa, x0, n * sizeof(T), cudaMemcpyDeviceToDevice, st));
  else { count_launch(); k_fill<T><<<grid_for(n, ctx->nsm), 256, 0, st>>>(n, L.xa, 0.0); }
  *iters = E.lsqr(L, solver, gamma, o.lsqr_warm_start ? L.xa : nullptr);
  // x_out = x0 + delta (no auxiliary update: copy, then add)
  const int g = grid_for(n, ctx->nsm);
  { count_launch(); k_outer_update<T><<<g, 256, 0, st>>>(m, -1, o.lsqr_warm_start, L.xa, L.dlt, (T*)x_out, L.a0x, L.a0y, L.a1x,
                                       L.a1y, 0, 0, 0, E.d_part, E.d_cnt + 4, E.d_box); }
  CK(cudaGetLastError());
}

extern "C" db_status db_lsqr_solve(db_context* ctx, const double* psf_host, int S, int m, db_solver solver, double gamma,
                        const void* b, const void* x0, const void* aux0, const void* aux1, void* x_out,
                        const db_opts* opts, int* iters, db_precision prec, db_stream stream) {
  if (!ctx) return DB_EINVAL;
  CountScope count_scope(ctx);
  try {
    REQUIRE(psf_host && b && x_out && iters, "null pointer argument");
    validate(m, S, 1, DB_HAAR);
    REQUIRE(gamma > 0, "gamma must be positive");
    db_opts o;
    db_default_opts(&o, nullptr);
    if (opts) o = *opts;
    CK(cudaSetDevice(ctx->device));
    cudaStream_t st = (cudaStream_t)stream;
    if (prec == DB_PREC_FP64) op_lsqr<double>(ctx, st, psf_host, S, m, solver, gamma, b, x0, aux0, aux1, x_out, o, iters);
    else if (prec == DB_PREC_FP32) op_lsqr<float>(ctx, st, psf_host, S, m, solver, gamma, b, x0, aux0, aux1, x_out, o, iters);
    else REQUIRE(false, "FP64 or FP32 only");
    CK(cudaStreamSynchronize(st));
    return DB_OK;
  } catch (DbError& e) {
    ctx->err = e.msg;
    return e.st;
  }
}

template <typename T>
static void op_gcv(db_context* ctx, cudaStream_t st, const double* psf_host, int S, int m, db_solver solver,
                   const void* b, const void* aux0, const void* aux1, const db_gcv_opts& g, double* gamma_out) {
  Engine<T> E(ctx, st);
  db_default_opts(&E.o, nullptr);
  E.go = g;
  ctx->arena.ensure(Engine<T>::footprint(m, 1, S, g));
  ctx->arena.reset();
  double* dpsf = ctx->arena.take<double>((size_t)S * S);
  CK(cudaMemcpyAsync(dpsf, psf_host, (size_t)S * S * sizeof(double), cudaMemcpyHostToDevice, st));
  E.build(dpsf, S, m, 1, DB_HAAR, nullptr, true);
  Level<T>& L = E.H.lv[0];
  const size_t n = L.n;
  CK(cudaMemcpyAsync(L.b, b, n * sizeof(T), cudaMemcpyDeviceToDevice, st));
  const T* a0 = (const T*)aux0;
  const T* a1 = (const T*)aux1;
  if (a0) {
    CK(cudaMemcpyAsync(L.a0x, a0, n * sizeof(T), cudaMemcpyDeviceToDevice, st));
    CK(cudaMemcpyAsync(L.a0y, a0 + n, n * sizeof(T), cudaMemcpyDeviceToDevice, st));
  }
  if (a1) {
    CK(cudaMemcpyAsync(L.a1x, a1, n * sizeof(T), cudaMemcpyDeviceToDevice, st));
    CK(cudaMemcpyAsync(L.a1y, a1 + n, n * sizeof(T), cudaMemcpyDeviceToDevice, st));
  } else {
    { count_launch(); k_fill<T><<<grid_for(n, ctx->nsm), 256, 0, st>>>(n, L.a1x, 0.0); }
    { count_launch(); k_fill<T><<<grid_for(n, ctx->nsm), 256, 0, st>>>(n, L.a1y, 0.0); }
  }
  const bool weighted = (solver == DB_IRLS) && a0;
  const bool shifted = (solver != DB_IRLS) && a0;
  *gamma_out = E.gcv(L, solver, weighted, shifted);
  E.check_blur_err();
}

extern "C" db_status db_gcv_select(db_context* ctx, const double* psf_host, int S, int m, db_solver solver, const void* b,
                        const void* aux0, const void* aux1, const db_gcv_opts* gcv, double* gamma_out,
                        db_precision prec, db_stream stream) {
  if (!ctx) return DB_EINVAL;
  CountScope count_scope(ctx);
  try {
    REQUIRE(psf_host && b && gamma_out, "null pointer argument");
    validate(m, S, 1, DB_HAAR);
    db_gcv_opts g;
    db_default_opts(nullptr, &g);
    if (gcv) g = *gcv;
    CK(cudaSetDevice(ctx->device));
    cudaStream_t st = (cudaStream_t)stream;
    if (prec == DB_PREC_FP64) op_gcv<double>(ctx, st, psf_host, S, m, solver, b, aux0, aux1, g, gamma_out);
    else if (prec == DB_PREC_FP32) op_gcv<float>(ctx, st, psf_host, S, m, solver, b, aux0, aux1, g, gamma_out);
    else REQUIRE(false, "FP64 or FP32 only");
    CK(cudaStreamSynchronize(st));
    return DB_OK;
  } catch (DbError& e) {
    ctx->err = e.msg;
    return e.st;
  }
}


// ============================================================================
// LSQR solve with a static workspace (no device allocation)
// ============================================================================
// db_lsqr_solve keeps its workspace in the context's arena, which grows with
// cudaMalloc. Some callers must not allocate device memory when they call:
// a process that hands all of HBM to its own memory pool at start-up (so a
// later cudaMalloc fails or would steal from the pool), or a latency-bound
// loop that may not take the allocator's synchronisation and fragmentation
// risk per call. db_lsqr_solve_static serves them from one fixed array that
// the module reserves when it is loaded, so the call allocates nothing.
// The array is shared by every call on a device: calls that overlap in time
// (two host threads, or two streams) race on it and must be serialised by
// the caller. The first call on a device looks the array up once
// (cudaGetSymbolAddress); make it before any stream capture begins.
constexpr size_t NOALLOC_BYTES = (size_t)16 << 20;   // 16 MiB
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_BYTES];

// Device address of the scratch array on the current device, looked up once
// per device.
static void* noalloc_base() {
  static std::mutex mu;
  static void* base[128] = {};
  int dev = 0;
  CK(cudaGetDevice(&dev));
  REQUIRE(dev >= 0 && dev < 128, "device ordinal out of range");
  std::lock_guard<std::mutex> lk(mu);
  if (!base[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      throw DbError{DB_ECUDA, std::string("cudaGetSymbolAddress of the static workspace failed: ") +
                                  cudaGetErrorString(e)};
    }
    base[dev] = p;
  }
  return base[dev];
}

// Bump allocator over the static array; running past its end is an input
// error (the problem is too large for this entry point), not an allocation.
struct StaticCursor {
  char* base;
  size_t off = 0;
  template <typename X> X* take(size_t count) {
    const size_t bytes = (count * sizeof(X) + 255) & ~size_t(255);
    if (off + bytes > NOALLOC_BYTES)
      throw DbError{DB_EINVAL, "problem too large for the 16 MiB static workspace of db_lsqr_solve_static"};
    X* p = reinterpret_cast<X*>(base + off);
    off += bytes;
    return p;
  }
};

template <typename T>
static void static_lsqr(cudaStream_t st, const double* psf_host, int S, int m, db_solver solver, double gamma,
                        const void* b, const void* x0, const void* aux0, const void* aux1, void* x_out,
                        const db_opts& o, int* iters) {
  using Acc = typename Traits<T>::Acc;
  int dev = 0, nsm = 0;
  CK(cudaGetDevice(&dev));
  CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  StaticCursor cur{static_cast<char*>(noalloc_base())};
  const size_t n = (size_t)m * m;
  // PSF factorisation (separable terms) into the workspace
  double* dpsf = cur.take<double>((size_t)S * S);
  double* wk = cur.take<double>((size_t)2 * S * S + S);
  double* fr = cur.take<double>((size_t)S * S);
  double* fc = cur.take<double>((size_t)S * S);
  int* d_nt = cur.take<int>(1);
  CK(cudaMemcpyAsync(dpsf, psf_host, (size_t)S * S * sizeof(double), cudaMemcpyHostToDevice, st));
  k_psf_svd<<<1, 256, 0, st>>>(S, dpsf, 1e-13, d_nt, fr, fc, wk);
  CK(cudaGetLastError());
  int nterms = 0;
  CK(cudaMemcpyAsync(&nterms, d_nt, sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  REQUIRE(nterms >= 1, "PSF is zero");
  // Every remaining piece of the workspace is carved out before the next
  // launch, so an input too large for the array is rejected (DB_EINVAL)
  // while no kernel of this call is in flight.
  Level<T> L;
  L.m = m;
  L.n = n;
  L.dlo = -(S / 2);
  L.w = S;
  const size_t nb = (size_t)nterms * m * S;
  L.Bd_r = cur.take<double>(nb);
  L.Bd_c = cur.take<double>(nb);
  L.br = cur.take<Acc>(nb); L.bc = cur.take<Acc>(nb); L.brT = cur.take<Acc>(nb); L.bcT = cur.take<Acc>(nb);
  // LSQR vectors; the caller's b, x0 and auxiliary planes are read in place
  L.uA = cur.take<T>(n); L.uLx = cur.take<T>(n); L.uLy = cur.take<T>(n);
  L.v = cur.take<T>(n); L.wv = cur.take<T>(n); L.dlt = cur.take<T>(n);
  const T* a0 = static_cast<const T*>(aux0);
  const T* a1 = static_cast<const T*>(aux1);
  const bool need_ones = !a0 && solver == DB_IRLS;                     // unit IRLS weights
  const bool need_zeros = (!a0 && solver != DB_IRLS) || !a1 || !x0;    // planes the caller left out
  T* ones = need_ones ? cur.take<T>(n) : nullptr;
  T* zeros = need_zeros ? cur.take<T>(n) : nullptr;
  // LSQR control block; the state, coefficients, tile counters and the grid
  // barrier must start at zero
  const int nt = L.ntiles_side();
  const int ntiles = nt * nt;
  double* d_part = cur.take<double>((size_t)std::max(ntiles * 6 + 64, 2 * 8 * nsm));
  unsigned* d_cnt = cur.take<unsigned>(64);
  double* d_box = cur.take<double>(64);
  GridBarrier* d_gb = cur.take<GridBarrier>(1);
  LsqrState* d_st = cur.take<LsqrState>(1);
  LsqrCoef<Acc>* d_coef = cur.take<LsqrCoef<Acc>>(1);
  LsqrProb<T, Acc>* d_prob = cur.take<LsqrProb<T, Acc>>(1);
  int* d_tile_prob = cur.take<int>(ntiles);
  // level-0 bands (zero-boundary blur, Sec. 5)
  const int gb = grid_for(nb, nsm);
  k_fine_bands_d<<<gb, 256, 0, st>>>(m, S, nterms, fr, L.Bd_r);
  k_fine_bands_d<<<gb, 256, 0, st>>>(m, S, nterms, fc, L.Bd_c);
  k_transpose_band<Acc><<<gb, 256, 0, st>>>(m, L.dlo, L.w, nterms, L.Bd_r, L.br, L.brT);
  k_transpose_band<Acc><<<gb, 256, 0, st>>>(m, L.dlo, L.w, nterms, L.Bd_c, L.bc, L.bcT);
  CK(cudaGetLastError());
  const int gn = grid_for(n, nsm);
  if (ones) k_fill<T><<<gn, 256, 0, st>>>(n, ones, 1.0);
  if (zeros) k_fill<T><<<gn, 256, 0, st>>>(n, zeros, 0.0);
  if (a0) { L.a0x = const_cast<T*>(a0); L.a0y = const_cast<T*>(a0) + n; }
  else if (solver == DB_IRLS) { L.a0x = L.a0y = ones; }
  else { L.a0x = L.a0y = zeros; }
  if (a1) { L.a1x = const_cast<T*>(a1); L.a1y = const_cast<T*>(a1) + n; }
  else { L.a1x = L.a1y = zeros; }
  const T* xstart = x0 ? static_cast<const T*>(x0) : zeros;
  CK(cudaGetLastError());
  CK(cudaMemsetAsync(d_cnt, 0, 64 * sizeof(unsigned), st));
  CK(cudaMemsetAsync(d_gb, 0, sizeof(GridBarrier), st));
  CK(cudaMemsetAsync(d_st, 0, sizeof(LsqrState), st));
  CK(cudaMemsetAsync(d_coef, 0, sizeof(LsqrCoef<Acc>), st));
  CK(cudaMemsetAsync(d_tile_prob, 0, sizeof(int) * ntiles, st));   // every tile belongs to problem 0
  LsqrProb<T, Acc> P{};
  P.op = L.op(nterms);
  P.m = m;
  P.solver = solver;
  P.gamma = gamma;
  P.sg = (Acc)std::sqrt(gamma);
  P.b = static_cast<const T*>(b);
  P.x0 = o.lsqr_warm_start ? xstart : nullptr;
  P.a0x = L.a0x; P.a0y = L.a0y; P.a1x = L.a1x; P.a1y = L.a1y;
  P.uA = L.uA; P.uLx = L.uLx; P.uLy = L.uLy; P.v = L.v; P.w = L.wv; P.dlt = L.dlt;
  P.nt = nt;
  P.ntiles = ntiles;
  P.tile_begin = 0;
  CK(cudaMemcpyAsync(d_prob, &P, sizeof(P), cudaMemcpyHostToDevice, st));
  LsqrCtl c;
  c.atol = o.lsqr_atol; c.btol = o.lsqr_btol; c.conlim = o.lsqr_conlim; c.maxit = o.lsqr_maxit;
  c.nprob = 1; c.ntiles = ntiles;
  c.tile_prob = d_tile_prob; c.part = d_part; c.cnt = d_cnt; c.st = d_st; c.gb = d_gb; c.coef = d_coef;
  c.limit_ns = (unsigned long long)o.barrier_timeout_us * 1000ull;
  c.band_cache = 0;
  c.band_pw = 0;
  c.cache_off = 0;
  TileGeom g0 = tile_geom(P.op, false), g1 = tile_geom(P.op, true);
  const int sm = std::max(tile_smem_elems(g0.H, g0.w), tile_smem_elems(g1.H, g1.w)) * (int)sizeof(Acc);
  auto kfn = k_lsqr<T, Acc>;
  require_smem_limit((const void*)kfn, sm);
  int per_sm = 0;
  CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kfn, 256, sm));
  REQUIRE(per_sm >= 1, "LSQR kernel does not fit on an SM");
  const int grid = std::max(1, std::min(ntiles, per_sm * nsm));
  const LsqrProb<T, Acc>* pp = d_prob;
  void* args[] = {(void*)&pp, (void*)&c};
  CK(cudaLaunchCooperativeKernel((const void*)kfn, dim3(grid), dim3(32, TY), args, sm, st));
  // x_out = x0 + delta
  k_outer_update<T><<<gn, 256, 0, st>>>(m, -1, o.lsqr_warm_start, xstart, L.dlt, static_cast<T*>(x_out), nullptr,
                                        nullptr, nullptr, nullptr, 0, 0, 0, d_part, d_cnt + 4, d_box);
  CK(cudaGetLastError());
  LsqrState S_;
  GridBarrier gbh;
  CK(cudaMemcpyAsync(&S_, d_st, sizeof(S_), cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(&gbh, d_gb, sizeof(gbh), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (gbh.error) throw DbError{DB_ETIMEOUT, "LSQR grid barrier timed out"};
  *iters = S_.its;
}

extern "C" db_status db_lsqr_solve_static(const double* psf_host, int S, int m, db_solver solver, double gamma,
                                          const void* b, const void* x0, const void* aux0, const void* aux1,
                                          void* x_out, const db_opts* opts, int* iters, db_precision prec,
                                          db_stream stream) {
  try {
    REQUIRE(psf_host && b && x_out && iters, "null pointer argument");
    validate(m, S, 1, DB_HAAR);
    REQUIRE(m <= 256, "db_lsqr_solve_static takes images of at most 256 x 256 pixels");
    REQUIRE(S <= 31, "db_lsqr_solve_static takes PSFs of at most 31 x 31");
    REQUIRE(solver == DB_IRLS || solver == DB_MM || solver == DB_SB, "unknown solver");
    REQUIRE(gamma > 0, "gamma must be positive");
    db_opts o;
    db_default_opts(&o, nullptr);
    if (opts) o = *opts;
    cudaStream_t st = (cudaStream_t)stream;
    if (prec == DB_PREC_FP64) static_lsqr<double>(st, psf_host, S, m, solver, gamma, b, x0, aux0, aux1, x_out, o, iters);
    else if (prec == DB_PREC_FP32) static_lsqr<float>(st, psf_host, S, m, solver, gamma, b, x0, aux0, aux1, x_out, o, iters);
    else REQUIRE(false, "FP64 or FP32 only");
    return DB_OK;
  } catch (DbError& e) {
    // kernels of this call may already be queued: wait for them, so that the
    // static array is idle when the error returns (the documented contract)
    cudaStreamSynchronize((cudaStream_t)stream);
    cudaGetLastError();
    g_last_error = e.msg;
    return e.st;
  }
}
