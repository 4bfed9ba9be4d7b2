// Vector kernels, deterministic reductions and an exclusive scan.
#include "common.cuh"

#include <atomic>
#include <ctime>

namespace fs {

int g_verbose = 0;
static std::atomic<unsigned long long> g_launches{0};
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
unsigned long long launch_count() { return g_launches.load(); }
void add_launches(long long delta) {
  g_launches.fetch_add((unsigned long long)delta, std::memory_order_relaxed);
}

thread_local BlockCache *g_cache = nullptr;

void *BlockCache::take(size_t sz) {
  auto it = blocks.find(sz);
  if (it == blocks.end()) return nullptr;
  void *p = it->second;
  blocks.erase(it);
  bytes -= sz;
  return p;
}

void BlockCache::put(void *p, size_t sz) {
  blocks.emplace(sz, p);
  bytes += sz;
}

void BlockCache::flush() {
  for (auto &b : blocks) cudaFree(b.second);
  blocks.clear();
  bytes = 0;
}

void *device_alloc(size_t sz, BlockCache *cache) {
  if (cache)
    if (void *p = cache->take(sz)) return p;
  void *p = nullptr;
  cudaError_t e = cudaMalloc(&p, sz);
  if (e == cudaErrorMemoryAllocation && cache && cache->bytes) {
    (void)cudaGetLastError();   // kept blocks of other sizes go back first
    cache->flush();
    e = cudaMalloc(&p, sz);
  }
  if (e == cudaErrorMemoryAllocation) {
    (void)cudaGetLastError();
    throw Error(FC_OOM, "cudaMalloc of " + std::to_string(sz) + " bytes failed");
  }
  FS_CUDA(e);
  return p;
}

cudaEvent_t Profiler::get() {
  if (used == pool.size()) {
    cudaEvent_t e;
    FS_CUDA(cudaEventCreate(&e));
    pool.push_back(e);
  }
  return pool[used++];
}
void Profiler::start(int k, cudaStream_t s) {
  if (!on) return;
  open_[k] = get();
  FS_CUDA(cudaEventRecord(open_[k], s));
}
void Profiler::stop(int k, cudaStream_t s, double b) {
  if (!on || !open_[k]) return;
  cudaEvent_t e = get();
  FS_CUDA(cudaEventRecord(e, s));
  rec[k].push_back({open_[k], e});
  bytes[k].push_back(b);
  open_[k] = nullptr;
}
void Profiler::reset() {
  used = 0;
  for (int k = 0; k < PK_N; k++) { rec[k].clear(); bytes[k].clear(); open_[k] = nullptr; }
}
void Profiler::stats(int k, int64_t *launches, double *ms, double *b) {
  double t = 0.0, bb = 0.0;
  for (size_t i = 0; i < rec[k].size(); i++) {
    FS_CUDA(cudaEventSynchronize(rec[k][i].second));
    float x = 0.f;
    FS_CUDA(cudaEventElapsedTime(&x, rec[k][i].first, rec[k][i].second));
    t += x;
    bb += bytes[k][i];
  }
  if (launches) *launches = (int64_t)rec[k].size();
  if (ms) *ms = t;
  if (b) *b = bb;
}
Profiler::~Profiler() {
  for (auto e : pool) cudaEventDestroy(e);
}

static double wall_ms() {
  timespec ts;
  clock_gettime(CLOCK_MONOTONIC, &ts);
  return ts.tv_sec * 1e3 + ts.tv_nsec * 1e-6;
}
PhaseTimer::PhaseTimer(bool on_, cudaStream_t s_, const char *tag_) : on(on_), s(s_), t0(0), tag(tag_) {
  if (on) {
    cudaStreamSynchronize(s);
    t0 = wall_ms();
  }
}
void PhaseTimer::mark(const char *what) {
  if (!on) return;
  cudaStreamSynchronize(s);
  double t = wall_ms();
  fprintf(stderr, "[fracsolve] %s %-28s %9.2f ms\n", tag, what, t - t0);
  t0 = t;
}

void cuda_fail(cudaError_t e, const char *what, const char *file, int line) {
  char buf[512];
  snprintf(buf, sizeof(buf), "%s failed: %s (%s:%d)", what, cudaGetErrorString(e), file, line);
  if (e == cudaErrorMemoryAllocation) throw Error(FC_OOM, buf);
  throw Error(FC_CUDA_ERROR, buf);
}

// ---------------------------------------------------------------- scan
namespace {
constexpr int kScanThreads = 256;
constexpr int kScanPer = 8;
constexpr int kScanTile = kScanThreads * kScanPer;

__device__ inline int block_exclusive_scan(int v, int *smem, int *total) {
  // Hillis-Steele over warp sums
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) smem[wid] = x;
  __syncthreads();
  if (wid == 0) {
    int w = (lane < kScanThreads / 32) ? smem[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    if (lane < kScanThreads / 32) smem[lane] = w;
  }
  __syncthreads();
  int pre = (wid > 0 ? smem[wid - 1] : 0) + x - v;
  if (total) *total = smem[kScanThreads / 32 - 1];
  __syncthreads();
  return pre;
}

__global__ void scan_tile_sums(const int *in, int n, int *sums) {
  __shared__ int sm[32];
  int base = blockIdx.x * kScanTile;
  int s = 0;
  for (int k = 0; k < kScanPer; k++) {
    int i = base + k * kScanThreads + threadIdx.x;
    if (i < n) s += in[i];
  }
  int tot;
  block_exclusive_scan(s, sm, &tot);
  if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

__global__ void scan_sums_single(int *sums, int nb) {
  __shared__ int sm[32];
  __shared__ int carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int base = 0; base < nb; base += kScanThreads) {
    int i = base + threadIdx.x;
    int v = i < nb ? sums[i] : 0;
    int tot;
    int pre = block_exclusive_scan(v, sm, &tot);
    if (i < nb) sums[i] = carry + pre;
    __syncthreads();
    if (threadIdx.x == 0) carry += tot;
    __syncthreads();
  }
  if (threadIdx.x == 0) sums[nb] = carry;
}

__global__ void scan_tile_apply(const int *in, int n, const int *sums, int *out) {
  __shared__ int sm[32];
  int base = blockIdx.x * kScanTile + threadIdx.x * kScanPer;
  int v[kScanPer];
  int s = 0;
#pragma unroll
  for (int k = 0; k < kScanPer; k++) {
    int i = base + k;
    v[k] = i < n ? in[i] : 0;
    s += v[k];
  }
  int pre = block_exclusive_scan(s, sm, nullptr) + sums[blockIdx.x];
#pragma unroll
  for (int k = 0; k < kScanPer; k++) {
    int i = base + k;
    if (i < n) out[i] = pre;
    pre += v[k];
  }
}

__global__ void scan_write_total(const int *sums, int nb, int *out, int n) { out[n] = sums[nb]; }
}  // namespace

int64_t exclusive_scan(const int *d_in, int *d_out, int n, cudaStream_t s) {
  if (n <= 0) {
    FS_CUDA(cudaMemsetAsync(d_out, 0, sizeof(int), s));
    return 0;
  }
  int nb = (n + kScanTile - 1) / kScanTile;
  DBuf<int> sums(nb + 1);
  // tile sums are over contiguous chunks of kScanTile elements, but the apply
  // kernel reads thread-contiguous runs; both cover the same tile range.
  scan_tile_sums<<<nb, kScanThreads, 0, s>>>(d_in, n, sums.p);
  FS_LAUNCHED();
  scan_sums_single<<<1, kScanThreads, 0, s>>>(sums.p, nb);
  FS_LAUNCHED();
  scan_tile_apply<<<nb, kScanThreads, 0, s>>>(d_in, n, sums.p, d_out);
  FS_LAUNCHED();
  scan_write_total<<<1, 1, 0, s>>>(sums.p, nb, d_out, n);
  FS_LAUNCHED();
  int tot = 0;
  FS_CUDA(cudaMemcpyAsync(&tot, d_out + n, sizeof(int), cudaMemcpyDeviceToHost, s));
  FS_CUDA(cudaStreamSynchronize(s));
  return tot;
}

// ---------------------------------------------------------------- reductions
namespace {
template <typename T>
__global__ void dot_partial(const T *__restrict__ x, const T *__restrict__ y, int64_t n,
                            double *partials) {
  __shared__ double sm[32];
  double acc = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    acc += (double)x[i] * (double)y[i];
  acc = warp_sum(acc);
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) sm[wid] = acc;
  __syncthreads();
  if (wid == 0) {
    double v = lane < (int)(blockDim.x >> 5) ? sm[lane] : 0.0;
    v = warp_sum(v);
    if (lane == 0) partials[blockIdx.x] = v;
  }
}

__global__ void sum_partials(const double *partials, int np, double *out) {
  __shared__ double sm[32];
  double acc = 0.0;
  for (int i = threadIdx.x; i < np; i += blockDim.x) acc += partials[i];
  acc = warp_sum(acc);
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) sm[wid] = acc;
  __syncthreads();
  if (wid == 0) {
    double v = lane < (int)(blockDim.x >> 5) ? sm[lane] : 0.0;
    v = warp_sum(v);
    if (lane == 0) *out = v;
  }
}
}  // namespace

template <typename T>
void nrm2sq_dev(const T *x, int64_t n, double *d_out, cudaStream_t s, double *d_partials) {
  dot_partial<T><<<kRedBlocks, 256, 0, s>>>(x, x, n, d_partials);
  FS_LAUNCHED();
  sum_partials<<<1, 1024, 0, s>>>(d_partials, kRedBlocks, d_out);
  FS_LAUNCHED();
}

template <typename T>
double dot(const T *x, const T *y, int64_t n, cudaStream_t s, double *d_tmp) {
  // d_tmp: kRedBlocks + 1 doubles
  dot_partial<T><<<kRedBlocks, 256, 0, s>>>(x, y, n, d_tmp);
  FS_LAUNCHED();
  sum_partials<<<1, 1024, 0, s>>>(d_tmp, kRedBlocks, d_tmp + kRedBlocks);
  FS_LAUNCHED();
  double h = 0;
  FS_CUDA(cudaMemcpyAsync(&h, d_tmp + kRedBlocks, sizeof(double), cudaMemcpyDeviceToHost, s));
  FS_CUDA(cudaStreamSynchronize(s));
  return h;
}

// ---------------------------------------------------------------- vectors
namespace {
template <typename TO, typename TI>
__global__ void k_cast(TO *out, const TI *in, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (TO)in[i];
}
template <typename T>
__global__ void k_fill(T *out, T v, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = v;
}
template <typename T>
__global__ void k_axpby(T *y, const T *x, double a, double b, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    y[i] = (T)(a * (double)x[i] + b * (double)y[i]);
}
template <typename TZ, typename TX, typename TY>
__global__ void k_axpbyz(TZ *z, const TX *x, const TY *y, double a, double b, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    z[i] = (TZ)(a * (double)x[i] + b * (double)y[i]);
}
template <typename T>
__global__ void k_scale(T *y, const T *x, double a, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    y[i] = (T)(a * (double)x[i]);
}
constexpr int kVecThreads = 256;
inline int vec_blocks(int64_t n) { return blocks_for(n, kVecThreads, kSMs * 16); }
}  // namespace

template <typename TO, typename TI>
void cast(TO *out, const TI *in, int64_t n, cudaStream_t s) {
  if (n <= 0) return;
  k_cast<TO, TI><<<vec_blocks(n), kVecThreads, 0, s>>>(out, in, n);
  FS_LAUNCHED();
}
template <typename T>
void fill(T *out, T v, int64_t n, cudaStream_t s) {
  if (n <= 0) return;
  k_fill<T><<<vec_blocks(n), kVecThreads, 0, s>>>(out, v, n);
  FS_LAUNCHED();
}
template <typename T>
void axpby(T *y, const T *x, double a, double b, int64_t n, cudaStream_t s) {
  if (n <= 0) return;
  k_axpby<T><<<vec_blocks(n), kVecThreads, 0, s>>>(y, x, a, b, n);
  FS_LAUNCHED();
}
template <typename TZ, typename TX, typename TY>
void axpbyz(TZ *z, const TX *x, const TY *y, double a, double b, int64_t n, cudaStream_t s) {
  if (n <= 0) return;
  k_axpbyz<TZ, TX, TY><<<vec_blocks(n), kVecThreads, 0, s>>>(z, x, y, a, b, n);
  FS_LAUNCHED();
}
template <typename T>
void scale_to(T *y, const T *x, double a, int64_t n, cudaStream_t s) {
  if (n <= 0) return;
  k_scale<T><<<vec_blocks(n), kVecThreads, 0, s>>>(y, x, a, n);
  FS_LAUNCHED();
}

#define FS_INST_T(T)                                                          \
  template double dot<T>(const T *, const T *, int64_t, cudaStream_t, double *); \
  template void nrm2sq_dev<T>(const T *, int64_t, double *, cudaStream_t, double *); \
  template void fill<T>(T *, T, int64_t, cudaStream_t);                       \
  template void axpby<T>(T *, const T *, double, double, int64_t, cudaStream_t); \
  template void scale_to<T>(T *, const T *, double, int64_t, cudaStream_t);
FS_INST_T(float)
FS_INST_T(double)
template void fill<int>(int *, int, int64_t, cudaStream_t);
template void cast<float, double>(float *, const double *, int64_t, cudaStream_t);
template void cast<double, float>(double *, const float *, int64_t, cudaStream_t);
template void cast<double, double>(double *, const double *, int64_t, cudaStream_t);
template void cast<float, float>(float *, const float *, int64_t, cudaStream_t);
template void axpbyz<double, double, double>(double *, const double *, const double *, double, double, int64_t, cudaStream_t);
template void axpbyz<float, float, float>(float *, const float *, const float *, double, double, int64_t, cudaStream_t);
template void axpbyz<double, float, double>(double *, const float *, const double *, double, double, int64_t, cudaStream_t);
template void axpbyz<float, double, double>(float *, const double *, const double *, double, double, int64_t, cudaStream_t);

}  // namespace fs
