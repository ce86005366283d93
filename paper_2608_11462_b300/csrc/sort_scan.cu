// sort_scan.cu -- device exclusive scan and stable LSD radix sort of (key, value) pairs,
// used by the setup phase (Morton sort, random enumeration, neighbour grid), and the
// library's per-device stream-ordered memory pool with the allocation context that
// plans and call temporaries draw on.
#include <functional>
#include <mutex>
#include <set>

#include "phs_internal.cuh"

namespace phs {

cudaMemPool_t scratch_pool() {
    static std::mutex mu;
    static cudaMemPool_t pools[64] = {};
    int dev = 0;
    PHS_CUDA(cudaGetDevice(&dev));
    PHS_REQUIRE(dev >= 0 && dev < 64, PHS_ERR_CUDA, "device ordinal out of range for the scratch pool");
    std::lock_guard<std::mutex> g(mu);
    if (!pools[dev]) {
        cudaMemPoolProps props{};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t pool;
        PHS_CUDA(cudaMemPoolCreate(&pool, &props));
        uint64_t keep = 1ull << 30;
        PHS_CUDA(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep));
        pools[dev] = pool;
    }
    return pools[dev];
}

AllocCtx &alloc_ctx() {
    static thread_local AllocCtx ctx;
    return ctx;
}

// a non-blocking stream per device for releases made outside any allocation scope
static cudaStream_t free_stream() {
    static std::mutex mu;
    static cudaStream_t streams[64] = {};
    int dev = 0;
    PHS_CUDA(cudaGetDevice(&dev));
    PHS_REQUIRE(dev >= 0 && dev < 64, PHS_ERR_CUDA, "device ordinal out of range for the release stream");
    std::lock_guard<std::mutex> g(mu);
    if (!streams[dev]) PHS_CUDA(cudaStreamCreateWithFlags(&streams[dev], cudaStreamNonBlocking));
    return streams[dev];
}

void once_per_device(int id, const std::function<void()> &fn) {
    static std::mutex mu;
    static std::set<std::pair<int, int>> done;
    int dev = 0;
    PHS_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> g(mu);
    if (done.count({dev, id})) return;
    fn();
    done.insert({dev, id});
}

void dbuf_alloc(void **p, size_t bytes, bool *pooled, int64_t **acct) {
    const AllocCtx &c = alloc_ctx();
    *pooled = false;
    *acct = nullptr;
    if (c.on) {
        PHS_CUDA(cudaMallocFromPoolAsync(p, bytes, scratch_pool(), c.s));
        *pooled = true;
        if (c.bytes) {
            *c.bytes += (int64_t)bytes;
            *acct = c.bytes;
        }
    } else {
        PHS_CUDA(cudaMalloc(p, bytes));
    }
}

void dbuf_free(void *p, size_t bytes, bool pooled, int64_t *acct) {
    // release paths run in destructors: errors are not thrown from here
    if (pooled) {
        const AllocCtx &c = alloc_ctx();
        cudaStream_t st = nullptr;
        if (c.on) st = c.s;
        else {
            try {
                st = free_stream();
            } catch (...) {
                st = nullptr;
            }
        }
        cudaFreeAsync(p, st);
    } else {
        cudaFree(p);
    }
    if (acct) *acct -= (int64_t)bytes;
}

namespace {

constexpr int SCAN_T = 1024;
constexpr int SCAN_ITEMS = 4;
constexpr int SCAN_TILE = SCAN_T * SCAN_ITEMS;

__device__ __forceinline__ int warp_incl_scan(int v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int u = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += u;
    }
    return v;
}

// block-wide exclusive scan of one value per thread (blockDim a multiple of 32, <= 1024);
// the block total is returned through *tot
__device__ int block_excl_scan(int v, int *tot) {
    __shared__ int wsum[32];
    __shared__ int total_s;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int inc = warp_incl_scan(v);
    if (lane == 31) wsum[w] = inc;
    __syncthreads();
    if (w == 0) {
        const int nw = blockDim.x >> 5;
        int sv = lane < nw ? wsum[lane] : 0;
        int si = warp_incl_scan(sv);
        if (lane < nw) wsum[lane] = si - sv;
        if (lane == 31) total_s = si;
    }
    __syncthreads();
    int res = wsum[w] + inc - v;
    *tot = total_s;
    __syncthreads();  // wsum/total_s may be reused by the next call
    return res;
}

__global__ void scan_tile_sums(const int *in, int64_t n, int *sums) {
    int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
    int s = 0;
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; ++i)
        if (base + i < n) s += in[base + i];
    int tot;
    block_excl_scan(s, &tot);
    if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

// single block: exclusive scan of the tile sums in place, total to sums[ntiles]
__global__ void scan_sums(int *sums, int64_t ntiles) {
    __shared__ int carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int64_t b = 0; b < ntiles; b += SCAN_T) {
        int64_t i = b + threadIdx.x;
        int v = i < ntiles ? sums[i] : 0;
        int tot;
        int ex = block_excl_scan(v, &tot);
        int c = carry;
        if (i < ntiles) sums[i] = ex + c;
        __syncthreads();
        if (threadIdx.x == 0) carry = c + tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) sums[ntiles] = carry;
}

__global__ void scan_tiles(const int *in, int *out, int64_t n, const int *sums) {
    int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
    int v[SCAN_ITEMS];
    int s = 0;
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; ++i) {
        v[i] = base + i < n ? in[base + i] : 0;
        s += v[i];
    }
    int tot;
    int ex = block_excl_scan(s, &tot) + sums[blockIdx.x];
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; ++i) {
        if (base + i < n) out[base + i] = ex;
        ex += v[i];
    }
}

// ---------------------------------------------------------------- radix sort
constexpr int RS_T = 256;
constexpr int RS_ITEMS = 8;
constexpr int RS_TILE = RS_T * RS_ITEMS;
constexpr int RS_WARPS = RS_T / 32;

__global__ void rs_hist(const uint64_t *keys, int64_t n, int shift, int *hist, int ntiles) {
    __shared__ int h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    int64_t base = (int64_t)blockIdx.x * RS_TILE;
    for (int it = 0; it < RS_ITEMS; ++it) {
        int64_t i = base + it * RS_T + threadIdx.x;
        if (i < n) atomicAdd(&h[(keys[i] >> shift) & 255], 1);
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * ntiles + blockIdx.x] = h[threadIdx.x];
}

__global__ void rs_scatter(const uint64_t *kin, const int *vin, uint64_t *kout, int *vout, int64_t n,
                           int shift, const int *offs, int ntiles) {
    __shared__ int wcount[RS_WARPS][257];
    __shared__ int woff[RS_WARPS][257];
    __shared__ int base_d[256];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    base_d[threadIdx.x] = offs[(int64_t)threadIdx.x * ntiles + blockIdx.x];
    for (int j = threadIdx.x; j < RS_WARPS * 257; j += RS_T) (&wcount[0][0])[j] = 0;
    __syncthreads();
    const int64_t tile = (int64_t)blockIdx.x * RS_TILE;
    for (int it = 0; it < RS_ITEMS; ++it) {
        int64_t i = tile + it * RS_T + threadIdx.x;
        bool valid = i < n;
        uint64_t k = valid ? kin[i] : 0;
        int v = valid ? vin[i] : 0;
        int d = valid ? (int)((k >> shift) & 255) : 256;
        unsigned peers = __match_any_sync(0xffffffffu, d);
        int lrank = __popc(peers & ((1u << lane) - 1u));
        int leader = __ffs(peers) - 1;
        if (lane == leader) wcount[w][d] = __popc(peers);
        __syncthreads();
        {
            int dd = threadIdx.x;  // one thread per digit
            int acc = 0;
            for (int ww = 0; ww < RS_WARPS; ++ww) {
                int c = wcount[ww][dd];
                woff[ww][dd] = base_d[dd] + acc;
                acc += c;
                wcount[ww][dd] = 0;
            }
            base_d[dd] += acc;
        }
        __syncthreads();
        if (valid) {
            int pos = woff[w][d] + lrank;
            kout[pos] = k;
            vout[pos] = v;
        }
        __syncthreads();
    }
}

}  // namespace

int64_t exclusive_scan_i32(const int *in, int *out, int64_t n, cudaStream_t s) {
    int64_t ntiles = (n + SCAN_TILE - 1) / SCAN_TILE;
    if (ntiles < 1) ntiles = 1;
    SBuf<int> sums(ntiles + 1, s);
    scan_tile_sums<<<(unsigned)ntiles, SCAN_T, 0, s>>>(in, n, sums.get());
    PHS_LAUNCH_CHECK();
    scan_sums<<<1, SCAN_T, 0, s>>>(sums.get(), ntiles);
    PHS_LAUNCH_CHECK();
    if (n > 0) {
        scan_tiles<<<(unsigned)ntiles, SCAN_T, 0, s>>>(in, out, n, sums.get());
        PHS_LAUNCH_CHECK();
    }
    int total = 0;
    PHS_CUDA(cudaMemcpyAsync(&total, sums.get() + ntiles, sizeof(int), cudaMemcpyDeviceToHost, s));
    PHS_CUDA(cudaStreamSynchronize(s));
    return total;
}

void radix_sort_pairs(uint64_t *keys, int *vals, int64_t n, int bits, cudaStream_t s) {
    if (n <= 1) return;
    int ntiles = (int)((n + RS_TILE - 1) / RS_TILE);
    SBuf<uint64_t> k2(n, s);
    SBuf<int> v2(n, s);
    SBuf<int> hist((size_t)256 * ntiles, s), offs((size_t)256 * ntiles, s);
    uint64_t *ka = keys, *kb = k2.get();
    int *va = vals, *vb = v2.get();
    int passes = (bits + 7) / 8;
    for (int ps = 0; ps < passes; ++ps) {
        int shift = ps * 8;
        rs_hist<<<ntiles, RS_T, 0, s>>>(ka, n, shift, hist.get(), ntiles);
        PHS_LAUNCH_CHECK();
        exclusive_scan_i32(hist.get(), offs.get(), (int64_t)256 * ntiles, s);
        rs_scatter<<<ntiles, RS_T, 0, s>>>(ka, va, kb, vb, n, shift, offs.get(), ntiles);
        PHS_LAUNCH_CHECK();
        std::swap(ka, kb);
        std::swap(va, vb);
    }
    if (ka != keys) {
        PHS_CUDA(cudaMemcpyAsync(keys, ka, n * sizeof(uint64_t), cudaMemcpyDeviceToDevice, s));
        PHS_CUDA(cudaMemcpyAsync(vals, va, n * sizeof(int), cudaMemcpyDeviceToDevice, s));
    }
    PHS_CUDA(cudaStreamSynchronize(s));
}

}  // namespace phs
