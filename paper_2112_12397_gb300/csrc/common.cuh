// Shared device-side infrastructure: owned device buffers, BSR matrices,
// status handling, deterministic reductions and scans.
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <cstdint>
#include <cstdio>
#include <map>
#include <stdexcept>
#include <string>
#include <vector>

#include "../../include/fracsolve.h"

namespace fs {

struct Error : std::runtime_error {
  int code;
  Error(int c, const std::string &m) : std::runtime_error(m), code(c) {}
};

[[noreturn]] void cuda_fail(cudaError_t e, const char *what, const char *file, int line);

#define FS_CUDA(x)                                                   \
  do {                                                               \
    cudaError_t e_ = (x);                                            \
    if (e_ != cudaSuccess) ::fs::cuda_fail(e_, #x, __FILE__, __LINE__); \
  } while (0)
// every kernel launch is followed by FS_LAUNCHED(): checks the launch and
// counts it (fc_launch_count)
void count_launch();
unsigned long long launch_count();
void add_launches(long long delta);   // kernels replayed by a graph (+) or captured only (-)
#define FS_LAUNCHED()               \
  do {                              \
    ::fs::count_launch();           \
    FS_CUDA(cudaGetLastError());    \
  } while (0)
#define FS_REQUIRE(cond, code, msg)                 \
  do {                                              \
    if (!(cond)) throw ::fs::Error((code), (msg));  \
  } while (0)

// ---------------------------------------------------------------- buffers
// Device blocks released by a context are kept for its next allocations of
// the same size instead of going back to the driver: a repeated fc_setup
// (a Newton sequence, or the bench) then allocates and frees nothing, where
// cudaFree would synchronise the device and cudaMalloc pay a driver call for
// each of the hierarchy's buffers.  Every kernel of a context runs on its one
// stream, so a block reused by the same context is stream-ordered after its
// previous use.  The cache belongs to the context (the first member, freed
// last) and is the one a DBuf sees while that context's entry point runs
// (g_cache); allocations made outside a context call go to the driver.
struct BlockCache {
  std::multimap<size_t, void *> blocks;
  size_t bytes = 0;
  void *take(size_t sz);
  void put(void *p, size_t sz);
  void flush();   // returns every kept block to the driver
  ~BlockCache() { flush(); }
};
extern thread_local BlockCache *g_cache;
void *device_alloc(size_t sz, BlockCache *cache);   // throws Error(FC_OOM) when the device is full

struct CacheScope {   // g_cache for the duration of one entry point
  BlockCache *prev;
  explicit CacheScope(BlockCache *c) : prev(g_cache) { g_cache = c; }
  ~CacheScope() { g_cache = prev; }
};

template <typename T>
struct DBuf {
  T *p = nullptr;
  size_t n = 0;
  BlockCache *cache = nullptr;   // where p goes back on release (nullptr: the driver)
  DBuf() = default;
  explicit DBuf(size_t n_) { alloc(n_); }
  static size_t rounded(size_t n_) { return (n_ * sizeof(T) + 255) & ~size_t(255); }
  void alloc(size_t n_) {
    release();
    if (n_ == 0) return;
    cache = g_cache;
    p = static_cast<T *>(device_alloc(rounded(n_), cache));
    n = n_;
  }
  // grow-only reallocation (contents are not kept)
  void ensure(size_t n_) {
    if (n_ > n) alloc(n_);
  }
  void release() {
    if (p) {
      if (cache) cache->put(p, rounded(n));
      else cudaFree(p);
    }
    p = nullptr;
    n = 0;
    cache = nullptr;
  }
  ~DBuf() { release(); }
  DBuf(DBuf &&o) noexcept : p(o.p), n(o.n), cache(o.cache) { o.p = nullptr; o.n = 0; o.cache = nullptr; }
  DBuf &operator=(DBuf &&o) noexcept {
    if (this != &o) {
      release();
      p = o.p; n = o.n; cache = o.cache;
      o.p = nullptr; o.n = 0; o.cache = nullptr;
    }
    return *this;
  }
  DBuf(const DBuf &) = delete;
  DBuf &operator=(const DBuf &) = delete;
  T *data() const { return p; }
  size_t size() const { return n; }
};

// Non-owning view of a block sparse row matrix on the device.
template <typename T>
struct BsrView {
  int nbr = 0, nbc = 0, br = 0, bc = 0;
  int64_t nnzb = 0;
  const int *rp = nullptr;
  const int *ci = nullptr;
  const T *val = nullptr;
};

// Owned block sparse row matrix on the device; blocks row-major br x bc.
template <typename T>
struct Bsr {
  int nbr = 0, nbc = 0, br = 0, bc = 0;
  int64_t nnzb = 0;
  DBuf<int> rp, ci;
  DBuf<T> val;
  BsrView<T> view() const {
    BsrView<T> v;
    v.nbr = nbr; v.nbc = nbc; v.br = br; v.bc = bc; v.nnzb = nnzb;
    v.rp = rp.p; v.ci = ci.p; v.val = val.p;
    return v;
  }
  void shape(int nbr_, int nbc_, int br_, int bc_) {
    nbr = nbr_; nbc = nbc_; br = br_; bc = bc_;
  }
  int64_t bsz() const { return (int64_t)br * bc; }
};

// ---------------------------------------------------------------- profiling
// CUDA-event timing of selected kernels on the launching stream.
enum ProfKernel {
  PK_SMOOTH0 = 0, PK_JAC = 1, PK_CGS = 2, PK_VCYCLE = 3, PK_PREC = 4, PK_RESID0 = 5, PK_RESTRICT0 = 6,
  PK_PROLONG0 = 7, PK_COARSE0 = 8, PK_VCYCLE_P = 9, PK_N = 10
};
struct Profiler {
  bool on = false;
  std::vector<cudaEvent_t> pool;
  size_t used = 0;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> rec[PK_N];
  std::vector<double> bytes[PK_N];
  cudaEvent_t open_[PK_N] = {};
  cudaEvent_t get();
  void start(int k, cudaStream_t s);
  void stop(int k, cudaStream_t s, double bytes_alg);
  void reset();
  // sums over recorded launches (synchronises on the events)
  void stats(int k, int64_t *launches, double *ms, double *bytes_alg);
  ~Profiler();
};

// library diagnostics level (set from fc_options.verbose by fc_setup)
extern int g_verbose;

// NVTX range for the duration of a scope (visible in Nsight timelines; a
// no-op unless a tool is attached)
struct NvtxRange {
  explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange &) = delete;
  NvtxRange &operator=(const NvtxRange &) = delete;
};

// Wall-clock phase timer for setup diagnostics (verbose only): synchronises
// the stream at each mark.
struct PhaseTimer {
  bool on;
  cudaStream_t s;
  double t0;
  const char *tag;
  PhaseTimer(bool on_, cudaStream_t s_, const char *tag_);
  void mark(const char *what);
};

// ---------------------------------------------------------------- launch
constexpr int kSMs = 152;
inline int blocks_for(int64_t n, int threads, int cap = 65535 * 16) {
  int64_t b = (n + threads - 1) / threads;
  if (b < 1) b = 1;
  if (b > cap) b = cap;
  return (int)b;
}

// ---------------------------------------------------------------- utilities
// out[0..n]: exclusive prefix sum of in[0..n-1], out[n] = total.  Returns the
// total (synchronises the stream).
int64_t exclusive_scan(const int *d_in, int *d_out, int n, cudaStream_t s);

// Deterministic dot products: fixed grid and fixed reduction order.
template <typename T>
double dot(const T *x, const T *y, int64_t n, cudaStream_t s, double *d_tmp);
// sum of squares to a device scalar (no host sync)
template <typename T>
void nrm2sq_dev(const T *x, int64_t n, double *d_out, cudaStream_t s, double *d_partials);
constexpr int kRedBlocks = 1024;   // partial sums of the two-stage reductions

template <typename TO, typename TI>
void cast(TO *out, const TI *in, int64_t n, cudaStream_t s);
template <typename T>
void fill(T *out, T v, int64_t n, cudaStream_t s);
// y = a*x + b*y
template <typename T>
void axpby(T *y, const T *x, double a, double b, int64_t n, cudaStream_t s);
// z = a*x + b*y (z may alias y)
template <typename TZ, typename TX, typename TY>
void axpbyz(TZ *z, const TX *x, const TY *y, double a, double b, int64_t n, cudaStream_t s);
// y = s * x
template <typename T>
void scale_to(T *y, const T *x, double a, int64_t n, cudaStream_t s);

// 64-bit SplitMix64 counter generator (Steele, Lea, Flood 2014).
__host__ __device__ inline uint64_t sm64_mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}
__host__ __device__ inline uint64_t sm64_draw(uint64_t seed, uint64_t stream, uint64_t i) {
  const uint64_t g = 0x9E3779B97F4A7C15ULL;
  uint64_t key = sm64_mix(seed * g + stream);
  return sm64_mix(key + (i + 1) * g);
}
__host__ __device__ inline double sm64_uniform(uint64_t seed, uint64_t stream, uint64_t i) {
  return (double)(sm64_draw(seed, stream, i) >> 11) * (1.0 / 9007199254740992.0);
}

// Warp reduction (sum) over `width` lanes.
template <typename T, int W = 32>
__device__ inline T warp_sum(T v) {
#pragma unroll
  for (int o = W / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o, W);
  return v;
}

}  // namespace fs
