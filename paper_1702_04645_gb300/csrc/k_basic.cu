// k_basic.cu -- buffers, device-wide prefix sums and the per-graph kernels:
// validation, strengths (Section 2.4: s_i and m_w), community totals Sigma_C,
// compaction of community names, partition composition (Algorithm 1,
// C = C_t C) and the exact modularity numerator (Section 2.4, Q_w).
#include <atomic>
#include <chrono>
#include <mutex>
#include <cstdio>
#include <cstring>

#include "slm_internal.cuh"

namespace slm {

void fail(slm_status st, const std::string &msg) { throw Error{st, msg}; }

static std::atomic<unsigned long long> g_launches{0};
void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
unsigned long long launch_count() { return g_launches.load(); }

void check_cuda(cudaError_t e, const char *what, const char *file, int line) {
    if (e == cudaSuccess) return;
    char buf[512];
    snprintf(buf, sizeof buf, "%s failed at %s:%d: %s", what, file, line, cudaGetErrorString(e));
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        fail(SLM_ERR_OUT_OF_MEMORY, buf);
    }
    fail(SLM_ERR_CUDA, buf);
}

static thread_local MemAcct *t_acct = nullptr;
static std::mutex g_acct_mu;

void MemAcct::add(long long b) {
    std::lock_guard<std::mutex> lk(g_acct_mu);
    cur += b;
    if (cur > peak) peak = cur;
}

MemAcct *set_thread_acct(MemAcct *a) {
    MemAcct *old = t_acct;
    t_acct = a;
    return old;
}

static thread_local bool t_blocking = false;
static thread_local cudaEvent_t t_ev = nullptr;
static thread_local int t_ev_dev = -1;

void set_thread_blocking_sync(bool on) { t_blocking = on; }

void stream_sync(cudaStream_t st) {
    if (!t_blocking) {
        SLM_CUDA(cudaStreamSynchronize(st));
        return;
    }
    int dev = 0;
    SLM_CUDA(cudaGetDevice(&dev));
    if (!t_ev || t_ev_dev != dev) {
        if (t_ev) cudaEventDestroy(t_ev);
        t_ev = nullptr;
        SLM_CUDA(cudaEventCreateWithFlags(&t_ev, cudaEventBlockingSync | cudaEventDisableTiming));
        t_ev_dev = dev;
    }
    SLM_CUDA(cudaEventRecord(t_ev, st));
    SLM_CUDA(cudaEventSynchronize(t_ev));
}

static std::mutex g_pool_mu;
static cudaMemPool_t g_pool[64] = {};

cudaMemPool_t lib_pool() {
    int dev = 0;
    SLM_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) fail(SLM_ERR_CUDA, "device ordinal out of range");
    std::lock_guard<std::mutex> lk(g_pool_mu);
    if (!g_pool[dev]) {
        cudaMemPoolProps props = {};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t p = nullptr;
        SLM_CUDA(cudaMemPoolCreate(&p, &props));
        unsigned long long keep = ~0ull;  // keep freed blocks for reuse
        cudaError_t e = cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &keep);
        if (e != cudaSuccess) {
            cudaMemPoolDestroy(p);
            check_cuda(e, "cudaMemPoolSetAttribute", __FILE__, __LINE__);
        }
        g_pool[dev] = p;
    }
    return g_pool[dev];
}

void trim_pool() {
    std::lock_guard<std::mutex> lk(g_pool_mu);
    for (int d = 0; d < 64; d++)
        if (g_pool[d]) cudaMemPoolTrimTo(g_pool[d], 0);
}

static std::atomic<long long> g_alloc_fail_in{0};

void set_alloc_failure(long long k) { g_alloc_fail_in.store(k > 0 ? k : 0); }

static thread_local RunControl *t_run_control = nullptr;

RunControl *set_thread_run_control(RunControl *c) {
    RunControl *prev = t_run_control;
    t_run_control = c;
    return prev;
}

double steady_seconds() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

void check_run_control() {
    const RunControl *c = t_run_control;
    if (!c) return;
    if (c->cancel && c->cancel->load(std::memory_order_relaxed))
        fail(SLM_ERR_CANCELLED, "the request was cancelled");
    if (c->deadline > 0 && steady_seconds() > c->deadline)
        fail(SLM_ERR_DEADLINE, "the request passed its deadline");
}

void DevBuf::alloc(size_t bytes, cudaStream_t s) {
    release();
    s_ = s;
    if (bytes == 0) bytes = 16;
    // injected failure (slm_debug_fail_allocation): the countdown reaches 1
    for (long long k = g_alloc_fail_in.load(); k > 0;) {
        if (g_alloc_fail_in.compare_exchange_weak(k, k - 1)) {
            if (k == 1) fail(SLM_ERR_OUT_OF_MEMORY, "injected allocation failure (slm_debug_fail_allocation)");
            break;
        }
    }
    SLM_CUDA(cudaMallocFromPoolAsync(&p_, bytes, lib_pool(), s));
    bytes_ = bytes;
    acct_ = t_acct;
    if (acct_) acct_->add((long long)bytes_);
}

static thread_local bool t_release_default = false;
ReleaseOnDefaultStream::ReleaseOnDefaultStream() : prev(t_release_default) { t_release_default = true; }
ReleaseOnDefaultStream::~ReleaseOnDefaultStream() { t_release_default = prev; }

void DevBuf::release() {
    if (p_) cudaFreeAsync(p_, t_release_default ? cudaStream_t(0) : s_);
    if (p_ && acct_) acct_->add(-(long long)bytes_);
    p_ = nullptr;
    bytes_ = 0;
    acct_ = nullptr;
}

// One event per device marks the end of the last cooperative launch; a mutex
// keeps the wait/launch/record sequence of different threads apart.
static std::mutex g_coop_mu;
static cudaEvent_t g_coop_ev[64] = {};

void coop_before(cudaStream_t st) {
    g_coop_mu.lock();
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess && dev >= 0 && dev < 64 && g_coop_ev[dev])
        e = cudaStreamWaitEvent(st, g_coop_ev[dev], 0);
    if (e != cudaSuccess) {
        g_coop_mu.unlock();
        check_cuda(e, "cooperative launch ordering", __FILE__, __LINE__);
    }
}

void coop_after(cudaStream_t st) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess && dev >= 0 && dev < 64) {
        if (!g_coop_ev[dev]) e = cudaEventCreateWithFlags(&g_coop_ev[dev], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventRecord(g_coop_ev[dev], st);
    }
    g_coop_mu.unlock();
    if (e != cudaSuccess) check_cuda(e, "cooperative launch ordering", __FILE__, __LINE__);
}

// Each thread keeps one pinned block for its counters for as long as it
// lives: freeing pinned memory waits for the whole device, which would stall
// every other stream at the end of each run.
namespace {
struct PinnedCounters {
    long long *h = nullptr;
    ~PinnedCounters() {
        if (h) cudaFreeHost(h);
    }
};
thread_local PinnedCounters t_counters;
}  // namespace

HostCounters::HostCounters() {
    if (!t_counters.h) SLM_CUDA(cudaMallocHost(&t_counters.h, 64 * sizeof(long long)));
    h = t_counters.h;
}
HostCounters::~HostCounters() = default;

// ---------------------------------------------------------------------------
// Exclusive prefix sums: reduce tiles, scan the tile sums (recursively), then
// scan each tile with its offset.
// ---------------------------------------------------------------------------
constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

template <class T> __device__ T block_exclusive_scan(T v, T *total) {
    __shared__ T warp_tot[kScanThreads / kWarp];
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    T x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[wid] = x;
    __syncthreads();
    if (wid == 0) {
        T t = lane < kScanThreads / kWarp ? warp_tot[lane] : T(0);
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            T y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        if (lane < kScanThreads / kWarp) warp_tot[lane] = t;
    }
    __syncthreads();
    T warp_off = wid > 0 ? warp_tot[wid - 1] : T(0);
    if (total) *total = warp_tot[kScanThreads / kWarp - 1];
    __syncthreads();
    return warp_off + x - v;
}

template <class T> __global__ void k_psum_reduce(const T *in, long long n, T *tile_sums) {
    long long base = (long long)blockIdx.x * kScanTile;
    T acc = 0;
    for (int k = 0; k < kScanItems; k++) {
        long long i = base + (long long)k * kScanThreads + threadIdx.x;
        if (i < n) acc += in[i];
    }
    T tot;
    block_exclusive_scan<T>(acc, &tot);
    if (threadIdx.x == 0) tile_sums[blockIdx.x] = tot;
}

template <class T>
__global__ void k_psum_tile(const T *in, T *out, long long n, const T *tile_off) {
    __shared__ T buf[kScanTile];
    long long base = (long long)blockIdx.x * kScanTile;
    for (int k = 0; k < kScanItems; k++) {
        long long i = base + (long long)k * kScanThreads + threadIdx.x;
        buf[k * kScanThreads + threadIdx.x] = i < n ? in[i] : T(0);
    }
    __syncthreads();
    T loc[kScanItems];
    T acc = 0;
    for (int k = 0; k < kScanItems; k++) {
        loc[k] = buf[threadIdx.x * kScanItems + k];
        acc += loc[k];
    }
    T tot;
    T pre = block_exclusive_scan<T>(acc, &tot) + (tile_off ? tile_off[blockIdx.x] : T(0));
    for (int k = 0; k < kScanItems; k++) {
        buf[threadIdx.x * kScanItems + k] = pre;
        pre += loc[k];
    }
    __syncthreads();
    for (int k = 0; k < kScanItems; k++) {
        long long i = base + (long long)k * kScanThreads + threadIdx.x;
        if (i < n) out[i] = buf[k * kScanThreads + threadIdx.x];
    }
}

template <class T>
__global__ void k_psum_total(const T *last_in, const T *out, long long n, T *total) {
    if (threadIdx.x == 0 && blockIdx.x == 0) *total = out[n - 1] + *last_in;
}

template <class T>
static void scan_impl(const T *in, T *out, long long n, T *total_dev, cudaStream_t s) {
    if (n <= 0) {
        if (total_dev) SLM_CUDA(cudaMemsetAsync(total_dev, 0, sizeof(T), s));
        return;
    }
    long long tiles = (n + kScanTile - 1) / kScanTile;
    // the last input element is needed for the total; keep it when in == out
    DevBuf last;
    if (total_dev && in == out) {
        last.alloc(sizeof(T), s);
        SLM_CUDA(cudaMemcpyAsync(last.get(), in + n - 1, sizeof(T), cudaMemcpyDeviceToDevice, s));
    }
    if (tiles == 1) {
        k_psum_tile<T><<<1, kScanThreads, 0, s>>>(in, out, n, nullptr);
        SLM_LAUNCH_CHECK();
    } else {
        DevBuf sums(tiles * sizeof(T), s);
        k_psum_reduce<T><<<(unsigned)tiles, kScanThreads, 0, s>>>(in, n, sums.as<T>());
        SLM_LAUNCH_CHECK();
        scan_impl<T>(sums.as<T>(), sums.as<T>(), tiles, nullptr, s);
        k_psum_tile<T><<<(unsigned)tiles, kScanThreads, 0, s>>>(in, out, n, sums.as<T>());
        SLM_LAUNCH_CHECK();
    }
    if (total_dev) {
        const T *src_last = (in == out) ? last.as<T>() : in + n - 1;
        k_psum_total<T><<<1, 32, 0, s>>>(src_last, out, n, total_dev);
        SLM_LAUNCH_CHECK();
    }
}

void exclusive_scan_i32(const int32_t *in, int32_t *out, long long n, int32_t *total_dev,
                        cudaStream_t s) {
    scan_impl<int32_t>(in, out, n, total_dev, s);
}
void exclusive_scan_i64(const long long *in, long long *out, long long n, long long *total_dev,
                        cudaStream_t s) {
    scan_impl<long long>(in, out, n, total_dev, s);
}

// ---------------------------------------------------------------------------
// CSR validation, one thread per entry (row_ptr was checked on the host:
// rp[0] = 0, non-decreasing, rp[n] = nnz).  A warp covers 32 consecutive
// entries; lanes 0 and 31 find the rows of the first and last of them, and
// every lane searches its own row between the two, so a long row is spread
// over many warps instead of one.
// ---------------------------------------------------------------------------
namespace {
// the row r in [lo, hi] with rp[r] <= e < rp[r + 1] (e < rp[n])
__device__ __forceinline__ int row_of_entry(long long e, const int32_t *rp, int lo, int hi) {
    while (lo < hi) {
        const int mid = lo + (hi - lo + 1) / 2;
        if ((long long)rp[mid] <= e) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}
}  // namespace

__global__ void k_validate(int32_t n, long long nnz, const int32_t *rp, const int32_t *col,
                           const int32_t *w, int *bad) {
    const int lane = threadIdx.x & 31;
    for (long long base = ((long long)blockIdx.x * blockDim.x + threadIdx.x) & ~31ll; base < nnz;
         base += (long long)gridDim.x * blockDim.x) {
        const long long p = base + lane;
        const long long last = min(base + 31, nnz - 1);
        int r = 0;
        if (lane == 0 || lane == 31) r = row_of_entry(lane == 0 ? base : last, rp, 0, n - 1);
        const int rlo = __shfl_sync(0xffffffffu, r, 0), rhi = __shfl_sync(0xffffffffu, r, 31);
        int b = 0;
        if (p < nnz) {
            const int i = row_of_entry(p, rp, rlo, rhi);
            const int j = col[p];
            if (j < 0 || j >= n) {
                b |= 1;
            } else {
                if (p > rp[i] && col[p - 1] >= j) b |= 1;  // sorted, no duplicates
                const int wp = w ? w[p] : 1;
                if (wp <= 0) b |= 2;
                // W_ji must exist with the same weight
                int a = rp[j], c = rp[j + 1] - 1;
                int found = -1;
                while (a <= c) {
                    const int mid = (a + c) >> 1;
                    const int v = col[mid];
                    if (v == i) { found = mid; break; }
                    if (v < i) a = mid + 1;
                    else c = mid - 1;
                }
                if (found < 0 || (w ? w[found] : 1) != wp) b |= 4;
            }
        }
#pragma unroll
        for (int o = 16; o; o >>= 1) b |= __shfl_xor_sync(0xffffffffu, b, o);
        if (lane == 0 && b) atomicOr(bad, b);
    }
}

int validate_csr(int32_t n, long long nnz, const int32_t *rp, const int32_t *col, const int32_t *w,
                 cudaStream_t s) {
    DevBuf bad(sizeof(int), s);
    SLM_CUDA(cudaMemsetAsync(bad.get(), 0, sizeof(int), s));
    if (n > 0 && nnz > 0) {
        k_validate<<<grid_for(nnz, 256), 256, 0, s>>>(n, nnz, rp, col, w, bad.as<int>());
        SLM_LAUNCH_CHECK();
    }
    int h = 0;
    SLM_CUDA(cudaMemcpyAsync(&h, bad.get(), sizeof(int), cudaMemcpyDeviceToHost, s));
    slm::stream_sync(s);
    return h;
}

// Number of entries of x outside [0, n).
__global__ void k_out_of_range(long long cnt, const int32_t *x, int32_t n, int *bad) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < cnt;
         i += (long long)gridDim.x * blockDim.x)
        if (x[i] < 0 || x[i] >= n) atomicAdd(bad, 1);
}

int count_out_of_range(long long cnt, const int32_t *x, int32_t n, cudaStream_t s) {
    if (cnt <= 0) return 0;
    DevBuf bad(sizeof(int), s);
    SLM_CUDA(cudaMemsetAsync(bad.get(), 0, sizeof(int), s));
    k_out_of_range<<<grid_for(cnt, 256), 256, 0, s>>>(cnt, x, n, bad.as<int>());
    SLM_LAUNCH_CHECK();
    int h = 0;
    SLM_CUDA(cudaMemcpyAsync(&h, bad.get(), sizeof(int), cudaMemcpyDeviceToHost, s));
    slm::stream_sync(s);
    return h;
}

// ---------------------------------------------------------------------------
// Strengths: s_i = sum_j W_ij, m_w = sum_i s_i (Section 2.4).
// ---------------------------------------------------------------------------
__global__ void k_strengths(int32_t n, const int32_t *rp, const int32_t *w, int32_t *s,
                            unsigned long long *m) {
    int lane = threadIdx.x & 31;
    long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    unsigned long long local = 0;
    for (long long i = warp; i < n; i += nwarps) {
        long long acc = 0;
        for (int p = rp[i] + lane; p < rp[i + 1]; p += 32) acc += w[p];
#pragma unroll
        for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) {
            s[i] = (int32_t)(acc > 0x7fffffffLL ? 0x7fffffff : acc);
            local += (unsigned long long)acc;
        }
    }
    if (lane == 0 && local) atomicAdd(m, local);
}

long long strengths(int32_t n, const int32_t *rp, const int32_t *w, int32_t *s_out,
                    cudaStream_t s) {
    DevBuf m(sizeof(unsigned long long), s);
    SLM_CUDA(cudaMemsetAsync(m.get(), 0, sizeof(unsigned long long), s));
    if (n > 0) {
        k_strengths<<<grid_for((long long)n * 32, 256), 256, 0, s>>>(n, rp, w, s_out,
                                                                     m.as<unsigned long long>());
        SLM_LAUNCH_CHECK();
    }
    unsigned long long h = 0;
    SLM_CUDA(cudaMemcpyAsync(&h, m.get(), sizeof h, cudaMemcpyDeviceToHost, s));
    slm::stream_sync(s);
    return (long long)h;
}

// ---------------------------------------------------------------------------
// Sigma_C = sum of s over the community named C.
// ---------------------------------------------------------------------------
// One add per community and warp: the lanes of a warp that share a community
// sum their strengths first (a community of a large share of the graph would
// otherwise take one atomic per member on one address).
__global__ void k_sigma(int32_t n, const int32_t *root, const int32_t *s, int32_t *sigma) {
    const int lane = threadIdx.x & 31;
    for (long long base = ((long long)blockIdx.x * blockDim.x + threadIdx.x) & ~31ll; base < n;
         base += (long long)gridDim.x * blockDim.x) {
        const long long v = base + lane;
        int sv = 0, r = 0;
        if (v < n) {
            sv = s[v];
            r = root[v];
        }
        const unsigned act = __ballot_sync(0xffffffffu, sv != 0);
        if (sv != 0) {
            const unsigned grp = __match_any_sync(act, r);
            const int sum = __reduce_add_sync(grp, sv);
            if (lane == __ffs(grp) - 1) atomicAdd(&sigma[r], sum);
        }
    }
}

void community_sigma(int32_t n, const int32_t *root, const int32_t *s, int32_t *sigma,
                     cudaStream_t st) {
    if (n <= 0) return;
    SLM_CUDA(cudaMemsetAsync(sigma, 0, sizeof(int32_t) * n, st));
    k_sigma<<<grid_for(n, 256), 256, 0, st>>>(n, root, s, sigma);
    SLM_LAUNCH_CHECK();
}

// packed (out, in) pairs: one 64-bit add sums both components (each stays below 2^30)
// (the lanes of a warp that share an index add their pairs first)
__global__ void k_sum_packed(int32_t n, const int32_t *idx, const unsigned long long *s,
                             unsigned long long *out) {
    const int lane = threadIdx.x & 31;
    for (long long base = ((long long)blockIdx.x * blockDim.x + threadIdx.x) & ~31ll; base < n;
         base += (long long)gridDim.x * blockDim.x) {
        const long long v = base + lane;
        unsigned long long sv = 0;
        int r = 0;
        if (v < n) {
            sv = s[v];
            r = idx[v];
        }
        const unsigned act = __ballot_sync(0xffffffffu, sv != 0);
        if (sv != 0) {
            const unsigned grp = __match_any_sync(act, r);
            unsigned long long sum = 0;
            // 64-bit sum over the group: its lanes read each other's values
            for (unsigned g = grp; g; g &= g - 1) sum += __shfl_sync(grp, sv, __ffs(g) - 1);
            if (lane == __ffs(grp) - 1) atomicAdd(&out[r], sum);
        }
    }
}

void community_sigma(int32_t n, const int32_t *root, const unsigned long long *s,
                     unsigned long long *sigma, cudaStream_t st) {
    if (n <= 0) return;
    SLM_CUDA(cudaMemsetAsync(sigma, 0, sizeof(unsigned long long) * n, st));
    k_sum_packed<<<grid_for(n, 256), 256, 0, st>>>(n, root, s, sigma);
    SLM_LAUNCH_CHECK();
}

void sum_strengths_by(int32_t n, const int32_t *id, const unsigned long long *s, int32_t K,
                      unsigned long long *out, cudaStream_t st) {
    if (K > 0) SLM_CUDA(cudaMemsetAsync(out, 0, sizeof(unsigned long long) * K, st));
    if (n <= 0) return;
    k_sum_packed<<<grid_for(n, 256), 256, 0, st>>>(n, id, s, out);
    SLM_LAUNCH_CHECK();
}

// ---------------------------------------------------------------------------
// Compaction: names in use (root[x] == x) ranked in increasing order.
// ---------------------------------------------------------------------------
__global__ void k_root_flags(int32_t n, const int32_t *root, int32_t *f) {
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (long long)gridDim.x * blockDim.x)
        f[v] = root[v] == v ? 1 : 0;
}
__global__ void k_gather_rank(int32_t n, const int32_t *root, const int32_t *rank, int32_t *id) {
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (long long)gridDim.x * blockDim.x)
        id[v] = rank[root[v]];
}

int32_t compact_labels(int32_t n, const int32_t *root, int32_t *id, int32_t *scratch_n,
                       cudaStream_t s) {
    if (n <= 0) return 0;
    DevBuf tot(sizeof(int32_t), s);
    k_root_flags<<<grid_for(n, 256), 256, 0, s>>>(n, root, scratch_n);
    SLM_LAUNCH_CHECK();
    exclusive_scan_i32(scratch_n, scratch_n, n, tot.as<int32_t>(), s);
    k_gather_rank<<<grid_for(n, 256), 256, 0, s>>>(n, root, scratch_n, id);
    SLM_LAUNCH_CHECK();
    int32_t K = 0;
    SLM_CUDA(cudaMemcpyAsync(&K, tot.get(), sizeof K, cudaMemcpyDeviceToHost, s));
    slm::stream_sync(s);
    return K;
}

__global__ void k_compose(int32_t n0, int32_t *comp, const int32_t *id) {
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < n0;
         v += (long long)gridDim.x * blockDim.x)
        comp[v] = id[comp[v]];
}

void compose_labels(int32_t n0, int32_t *comp, const int32_t *id, cudaStream_t s) {
    if (n0 <= 0) return;
    k_compose<<<grid_for(n0, 256), 256, 0, s>>>(n0, comp, id);
    SLM_LAUNCH_CHECK();
}

// ---------------------------------------------------------------------------
// Modularity numerator sum_C (m_w W_in(C) - Sigma_C^2), exact in 64 bits
// (both sums are below m_w^2 < 2^62).
// ---------------------------------------------------------------------------
__global__ void k_mod_accumulate(int32_t n, const int32_t *rp, const int32_t *col,
                                 const int32_t *w, const int32_t *labels,
                                 unsigned long long *win, unsigned long long *sig) {
    int lane = threadIdx.x & 31;
    long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long u = warp; u < n; u += nwarps) {
        int lu = labels[u];
        long long in = 0, su = 0;
        for (int p = rp[u] + lane; p < rp[u + 1]; p += 32) {
            su += w[p];
            if (labels[col[p]] == lu) in += w[p];
        }
#pragma unroll
        for (int o = 16; o; o >>= 1) {
            in += __shfl_xor_sync(0xffffffffu, in, o);
            su += __shfl_xor_sync(0xffffffffu, su, o);
        }
        if (lane == 0) {
            if (in) atomicAdd(&win[lu], (unsigned long long)in);
            if (su) atomicAdd(&sig[lu], (unsigned long long)su);
        }
    }
}

__global__ void k_mod_reduce(int32_t n, const unsigned long long *win,
                             const unsigned long long *sig, unsigned long long m,
                             unsigned long long *out2) {
    unsigned long long a = 0, b = 0;
    for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < n;
         c += (long long)gridDim.x * blockDim.x) {
        a += m * win[c];
        b += sig[c] * sig[c];
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        b += __shfl_xor_sync(0xffffffffu, b, o);
    }
    if ((threadIdx.x & 31) == 0) {
        if (a) atomicAdd(&out2[0], a);
        if (b) atomicAdd(&out2[1], b);
    }
}

long long modularity_num(int32_t n, const int32_t *rp, const int32_t *col, const int32_t *w,
                         const int32_t *labels, long long m_w, cudaStream_t s) {
    if (n <= 0 || m_w == 0) return 0;
    DevBuf win(sizeof(unsigned long long) * n, s), sig(sizeof(unsigned long long) * n, s),
        out(2 * sizeof(unsigned long long), s);
    SLM_CUDA(cudaMemsetAsync(win.get(), 0, win.bytes(), s));
    SLM_CUDA(cudaMemsetAsync(sig.get(), 0, sig.bytes(), s));
    SLM_CUDA(cudaMemsetAsync(out.get(), 0, out.bytes(), s));
    k_mod_accumulate<<<grid_for((long long)n * 32, 256), 256, 0, s>>>(
        n, rp, col, w, labels, win.as<unsigned long long>(), sig.as<unsigned long long>());
    SLM_LAUNCH_CHECK();
    k_mod_reduce<<<grid_for(n, 256, 1024), 256, 0, s>>>(n, win.as<unsigned long long>(),
                                                         sig.as<unsigned long long>(),
                                                         (unsigned long long)m_w,
                                                         out.as<unsigned long long>());
    SLM_LAUNCH_CHECK();
    unsigned long long h[2];
    SLM_CUDA(cudaMemcpyAsync(h, out.get(), sizeof h, cudaMemcpyDeviceToHost, s));
    slm::stream_sync(s);
    return (long long)h[0] - (long long)h[1];
}

// per label: internal U weight and the packed strength total
__global__ void k_modd_accumulate(int32_t n, const int32_t *rp, const int32_t *col,
                                  const int32_t *w, const unsigned long long *s2,
                                  const int32_t *labels, unsigned long long *win,
                                  unsigned long long *sig) {
    int lane = threadIdx.x & 31;
    long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long u = warp; u < n; u += nwarps) {
        int lu = labels[u];
        long long in = 0;
        for (int p = rp[u] + lane; p < rp[u + 1]; p += 32)
            if (labels[col[p]] == lu) in += w[p];
#pragma unroll
        for (int o = 16; o; o >>= 1) in += __shfl_xor_sync(0xffffffffu, in, o);
        if (lane == 0) {
            if (in) atomicAdd(&win[lu], (unsigned long long)in);
            if (s2[u]) atomicAdd(&sig[lu], s2[u]);
        }
    }
}

// out2[0] = m_w sum U_in, out2[1] = sum 2 Sigma^out Sigma^in (each below 2^62)
__global__ void k_modd_reduce(int32_t n, const unsigned long long *win,
                              const unsigned long long *sig, unsigned long long m,
                              unsigned long long *out2) {
    unsigned long long a = 0, b = 0;
    for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < n;
         c += (long long)gridDim.x * blockDim.x) {
        a += m * win[c];
        b += (unsigned long long)NMDir::cross((long long)sig[c], (long long)sig[c]);
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        b += __shfl_xor_sync(0xffffffffu, b, o);
    }
    if ((threadIdx.x & 31) == 0) {
        if (a) atomicAdd(&out2[0], a);
        if (b) atomicAdd(&out2[1], b);
    }
}

long long modularity_num_directed(int32_t n, const int32_t *rp, const int32_t *col,
                                  const int32_t *w, const unsigned long long *s2,
                                  const int32_t *labels, long long m_w, cudaStream_t s) {
    if (n <= 0 || m_w == 0) return 0;
    DevBuf win(sizeof(unsigned long long) * n, s), sig(sizeof(unsigned long long) * n, s),
        out(2 * sizeof(unsigned long long), s);
    SLM_CUDA(cudaMemsetAsync(win.get(), 0, win.bytes(), s));
    SLM_CUDA(cudaMemsetAsync(sig.get(), 0, sig.bytes(), s));
    SLM_CUDA(cudaMemsetAsync(out.get(), 0, out.bytes(), s));
    k_modd_accumulate<<<grid_for((long long)n * 32, 256), 256, 0, s>>>(
        n, rp, col, w, s2, labels, win.as<unsigned long long>(), sig.as<unsigned long long>());
    SLM_LAUNCH_CHECK();
    k_modd_reduce<<<grid_for(n, 256, 1024), 256, 0, s>>>(n, win.as<unsigned long long>(),
                                                          sig.as<unsigned long long>(),
                                                          (unsigned long long)m_w,
                                                          out.as<unsigned long long>());
    SLM_LAUNCH_CHECK();
    unsigned long long h[2];
    SLM_CUDA(cudaMemcpyAsync(h, out.get(), sizeof h, cudaMemcpyDeviceToHost, s));
    slm::stream_sync(s);
    // both terms are even: U counts every internal arc in both rows
    return ((long long)h[0] - (long long)h[1]) / 2;
}

double modularity_from_num(long long num, long long m_w) {
    if (m_w == 0) return 0.0;
    return (double)num / ((double)m_w * (double)m_w);
}

// ---------------------------------------------------------------------------
// Forests of graphs: one block-diagonal CSR, node ranges per graph.
// ---------------------------------------------------------------------------
__global__ void k_gid(int32_t n, const int32_t *goff, int32_t G, int32_t *gid) {
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (long long)gridDim.x * blockDim.x) {
        int lo = 0, hi = G - 1;  // last g with goff[g] <= v
        while (lo < hi) {
            int mid = (lo + hi + 1) >> 1;
            if (goff[mid] <= v) lo = mid;
            else hi = mid - 1;
        }
        gid[v] = lo;
    }
}

void graph_of_nodes(int32_t n, const int32_t *goff, int32_t G, int32_t *gid, cudaStream_t st) {
    if (n <= 0 || G <= 0) return;
    k_gid<<<grid_for(n, 256), 256, 0, st>>>(n, goff, G, gid);
    SLM_LAUNCH_CHECK();
}

__global__ void k_forest_check(int32_t n, const int32_t *rp, const int32_t *col, const int32_t *s,
                               const int32_t *gid, unsigned long long *mg,
                               unsigned long long *cross) {
    const int lane = threadIdx.x & 31;
    const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long u = warp; u < n; u += nwarps) {
        const int g = gid[u];
        unsigned c = 0;
        for (int p = rp[u] + lane; p < rp[u + 1]; p += 32) c += gid[col[p]] != g;
#pragma unroll
        for (int o = 16; o; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
        if (lane == 0) {
            if (c) atomicAdd(cross, (unsigned long long)c);
            if (s[u]) atomicAdd(&mg[g], (unsigned long long)s[u]);
        }
    }
}

long long forest_check_and_weights(int32_t n, const int32_t *rp, const int32_t *col,
                                   const int32_t *s, const int32_t *gid, int32_t G,
                                   long long *mg, cudaStream_t st) {
    DevBuf cross(8, st);
    SLM_CUDA(cudaMemsetAsync(cross.get(), 0, 8, st));
    SLM_CUDA(cudaMemsetAsync(mg, 0, 8 * (size_t)G, st));
    if (n > 0) {
        k_forest_check<<<grid_for((long long)n * 32, 256), 256, 0, st>>>(
            n, rp, col, s, gid, reinterpret_cast<unsigned long long *>(mg), cross.as<unsigned long long>());
        SLM_LAUNCH_CHECK();
    }
    unsigned long long h = 0;
    SLM_CUDA(cudaMemcpyAsync(&h, cross.get(), 8, cudaMemcpyDeviceToHost, st));
    slm::stream_sync(st);
    return (long long)h;
}

__global__ void k_roots_per_graph(int32_t n, const int32_t *root, const int32_t *gid, int32_t *Kg) {
    const int lane = threadIdx.x & 31;
    for (long long base = ((long long)blockIdx.x * blockDim.x + threadIdx.x) & ~31ll; base < n;
         base += (long long)gridDim.x * blockDim.x) {
        const long long v = base + lane;
        const bool isroot = v < n && root[v] == v;
        warp_count(Kg, isroot ? gid[v] : 0, isroot);
    }
}

void roots_per_graph(int32_t n, const int32_t *root, const int32_t *gid, int32_t *Kg,
                     cudaStream_t st) {
    if (n <= 0) return;
    k_roots_per_graph<<<grid_for(n, 256), 256, 0, st>>>(n, root, gid, Kg);
    SLM_LAUNCH_CHECK();
}

__global__ void k_cands_per_graph(int32_t n, const int32_t *gid, const int32_t *active,
                                  long long *gain, int32_t *cand_g) {
    const int lane = threadIdx.x & 31;
    for (long long base = ((long long)blockIdx.x * blockDim.x + threadIdx.x) & ~31ll; base < n;
         base += (long long)gridDim.x * blockDim.x) {
        const long long v = base + lane;
        int g = 0;
        bool cand = false;
        if (v < n && gain[v] > 0) {
            g = gid[v];
            if (!active[g]) gain[v] = 0;  // a graph that stopped keeps its partition
            else cand = true;
        }
        warp_count(cand_g, g, cand);
    }
}

void candidates_per_graph(int32_t n, const int32_t *gid, const int32_t *active, long long *gain,
                          int32_t *cand_g, cudaStream_t st) {
    if (n <= 0) return;
    k_cands_per_graph<<<grid_for(n, 256), 256, 0, st>>>(n, gid, active, gain, cand_g);
    SLM_LAUNCH_CHECK();
}

__global__ void k_modf_reduce(int32_t nlab, const unsigned long long *win,
                              const unsigned long long *sig, const int32_t *loff, int32_t G,
                              const long long *mg, unsigned long long *a, unsigned long long *b) {
    for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < nlab;
         c += (long long)gridDim.x * blockDim.x) {
        if (!win[c] && !sig[c]) continue;
        int lo = 0, hi = G - 1;  // graph owning label c
        while (lo < hi) {
            int mid = (lo + hi + 1) >> 1;
            if (loff[mid] <= c) lo = mid;
            else hi = mid - 1;
        }
        if (win[c]) atomicAdd(&a[lo], (unsigned long long)mg[lo] * win[c]);
        if (sig[c]) atomicAdd(&b[lo], sig[c] * sig[c]);
    }
}

__global__ void k_modf_finish(int32_t G, const unsigned long long *a, const unsigned long long *b,
                              long long *nums) {
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < G; g += gridDim.x * blockDim.x)
        nums[g] = (long long)a[g] - (long long)b[g];
}

void modularity_forest(int32_t n, const int32_t *rp, const int32_t *col, const int32_t *w,
                       const int32_t *labels, int32_t nlab, const int32_t *gid,
                       const int32_t *loff, int32_t G, const long long *mg, long long *nums,
                       cudaStream_t st) {
    (void)gid;
    if (G <= 0) return;
    const size_t L = (size_t)(nlab > 0 ? nlab : 1);
    DevBuf win(8 * L, st), sig(8 * L, st), a(8 * (size_t)G, st), b(8 * (size_t)G, st);
    SLM_CUDA(cudaMemsetAsync(win.get(), 0, 8 * L, st));
    SLM_CUDA(cudaMemsetAsync(sig.get(), 0, 8 * L, st));
    SLM_CUDA(cudaMemsetAsync(a.get(), 0, 8 * (size_t)G, st));
    SLM_CUDA(cudaMemsetAsync(b.get(), 0, 8 * (size_t)G, st));
    if (n > 0) {
        k_mod_accumulate<<<grid_for((long long)n * 32, 256), 256, 0, st>>>(
            n, rp, col, w, labels, win.as<unsigned long long>(), sig.as<unsigned long long>());
        SLM_LAUNCH_CHECK();
        k_modf_reduce<<<grid_for(nlab, 256), 256, 0, st>>>(
            nlab, win.as<unsigned long long>(), sig.as<unsigned long long>(), loff, G, mg,
            a.as<unsigned long long>(), b.as<unsigned long long>());
        SLM_LAUNCH_CHECK();
    }
    k_modf_finish<<<grid_for(G, 256), 256, 0, st>>>(G, a.as<unsigned long long>(),
                                                    b.as<unsigned long long>(), nums);
    SLM_LAUNCH_CHECK();
}

}  // namespace slm
