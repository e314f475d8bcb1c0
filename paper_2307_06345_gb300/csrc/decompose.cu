// Domain decomposition of a particle set spread over several processes (Sec. 6): the bounding
// cube of the union from per-axis bounds reduced over the processes, and the cut of the globally
// replicated cornerstone array into n_ranks bins of consecutive leaves holding about N_tot / n_ranks
// particles each. Independent of the key length (compiled once).
//
// Cut r (0 < r < n_ranks) is the first leaf i whose preceding leaves hold at least r N_tot / n_ranks
// particles, compared exactly as integers (prefix_i * n_ranks >= N_tot * r), n_l if none. The
// exclusive prefix of the counts is monotone, so cut r is the number of leaves with
// prefix_i * n_ranks < N_tot * r, i.e. with r0_i = floor(prefix_i * n_ranks / N_tot) + 1 <= r: a
// histogram of r0 over the leaves followed by a prefix sum over r gives every cut at once.
#include "common.cuh"

namespace cst {
namespace {

constexpr int kDecThreads = 256;
constexpr int kDecItems = 16;                        // consecutive leaves per thread
constexpr int kDecChunk = kDecThreads * kDecItems;  // leaves per block

__global__ void cube_from_bounds_kernel(const double* __restrict__ bounds, double* __restrict__ box) {
    if (threadIdx.x != 0) return;
    const double lo0 = bounds[0];
    if (isinf(lo0) && lo0 > 0.0) {  // no point on any process
        box[0] = box[1] = box[2] = 0.0;
        box[3] = 1.0;
        return;
    }
    double side = 0.0;
    for (int d = 0; d < 3; ++d) {
        box[d] = bounds[d];
        const double ext = __dsub_rn(bounds[3 + d], bounds[d]);
        side = ext > side ? ext : side;
    }
    box[3] = side > 0.0 ? side : 1.0;
}

// Sum of the counts of every chunk of kDecChunk leaves.
__global__ void __launch_bounds__(kDecThreads) dec_chunk_sum_kernel(const u32* __restrict__ N, long long nl,
                                                                    u64* __restrict__ chunk) {
    __shared__ u64 s_warp[kDecThreads / 32];
    const long long base = (long long)blockIdx.x * kDecChunk;
    u64 sum = 0;
#pragma unroll
    for (int k = 0; k < kDecItems; ++k) {
        const long long i = base + k * kDecThreads + threadIdx.x;
        if (i < nl) sum += N[i];
    }
    for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
    if ((threadIdx.x & 31) == 0) s_warp[threadIdx.x >> 5] = sum;
    __syncthreads();
    if (threadIdx.x == 0) {
        u64 t = 0;
        for (int w = 0; w < kDecThreads / 32; ++w) t += s_warp[w];
        chunk[blockIdx.x] = t;
    }
}

// Exclusive scan of the chunk sums in place (one block), and the total.
__global__ void __launch_bounds__(1024) dec_scan_kernel(u64* __restrict__ chunk, long long nchunks,
                                                        u64* __restrict__ total) {
    __shared__ u64 s_warp[32];
    const long long per = (nchunks + 1023) / 1024;
    const long long c0 = threadIdx.x * per, c1 = c0 + per < nchunks ? c0 + per : nchunks;
    u64 sum = 0;
    for (long long c = c0; c < c1; ++c) sum += chunk[c];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    u64 incl = sum;
    for (int o = 1; o < 32; o <<= 1) {
        const u64 t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) s_warp[warp] = incl;
    __syncthreads();
    u64 before = 0;
    for (int w = 0; w < warp; ++w) before += s_warp[w];
    if (threadIdx.x == 1023) *total = before + incl;
    u64 run = before + incl - sum;
    for (long long c = c0; c < c1; ++c) {
        const u64 v = chunk[c];
        chunk[c] = run;
        run += v;
    }
}

// Every leaf's r0 (from its exclusive prefix: the chunk's prefix plus the scan inside the chunk),
// counted into hist[1 .. n_ranks - 1]. A thread's leaves are consecutive, so their r0 do not
// decrease and each distinct value takes one atomic.
__global__ void __launch_bounds__(kDecThreads) dec_hist_kernel(const u32* __restrict__ N, long long nl,
                                                               const u64* __restrict__ chunk_prefix,
                                                               const u64* __restrict__ total_p, int n_ranks,
                                                               u32* __restrict__ hist) {
    __shared__ u64 s_warp[kDecThreads / 32];
    const u64 total = *total_p;
    if (total == 0) return;  // every inner cut stays 0
    const long long i0 = (long long)blockIdx.x * kDecChunk + (long long)threadIdx.x * kDecItems;
    u32 v[kDecItems];
    u64 sum = 0;
#pragma unroll
    for (int k = 0; k < kDecItems; ++k) {
        v[k] = i0 + k < nl ? N[i0 + k] : 0u;
        sum += v[k];
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    u64 incl = sum;
    for (int o = 1; o < 32; o <<= 1) {
        const u64 t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) s_warp[warp] = incl;
    __syncthreads();
    u64 before = 0;
    for (int w = 0; w < warp; ++w) before += s_warp[w];
    u64 prefix = chunk_prefix[blockIdx.x] + before + incl - sum;  // before leaf i0
    const u64 w = static_cast<u64>(n_ranks);
    u64 run_r = 0;
    u32 run_n = 0;
#pragma unroll
    for (int k = 0; k < kDecItems; ++k) {
        if (i0 + k >= nl) break;
        const u64 r0 = prefix * w / total + 1;
        if (r0 != run_r) {
            if (run_n && run_r < w) atomicAdd(hist + run_r, run_n);
            run_r = r0;
            run_n = 0;
        }
        ++run_n;
        prefix += v[k];
    }
    if (run_n && run_r < w) atomicAdd(hist + run_r, run_n);
}

// cuts[r] = hist[1] + ... + hist[r] for 0 < r < n_ranks; cuts[0] = 0, cuts[n_ranks] = n_l (one block).
__global__ void __launch_bounds__(1024) dec_cuts_kernel(const u32* __restrict__ hist, int n_ranks, long long nl,
                                                        long long* __restrict__ cuts) {
    __shared__ long long s_warp[32];
    const int per = (n_ranks + 1023) / 1024;
    const int r0 = threadIdx.x * per, r1 = min(r0 + per, n_ranks);
    long long sum = 0;
    for (int r = r0; r < r1; ++r) sum += r >= 1 ? hist[r] : 0u;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    long long incl = sum;
    for (int o = 1; o < 32; o <<= 1) {
        const long long t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) s_warp[warp] = incl;
    __syncthreads();
    long long run = 0;
    for (int w = 0; w < warp; ++w) run += s_warp[w];
    run += incl - sum;
    for (int r = r0; r < r1; ++r) {
        run += r >= 1 ? hist[r] : 0u;
        cuts[r] = r == 0 ? 0 : run;
    }
    if (threadIdx.x == 0) cuts[n_ranks] = nl;
}

struct DecLayout {
    u64* chunk;
    u64* total;
    u32* hist;
    long long nchunks;
    size_t bytes;
};

DecLayout dec_layout(void* ws, long long nl, int n_ranks) {
    DecLayout l;
    Carver c(ws);
    l.nchunks = (nl + kDecChunk - 1) / kDecChunk;
    l.chunk = c.take<u64>((size_t)(l.nchunks > 0 ? l.nchunks : 1));
    l.total = c.take<u64>(1);
    l.hist = c.take<u32>((size_t)n_ranks + 1);
    l.bytes = c.size();
    return l;
}

constexpr int kMaxRanks = 1 << 16;

}  // namespace
}  // namespace cst

extern "C" {

int cstone_cube_from_bounds(const double* bounds, double* box, void* stream) {
    if (!bounds || !box) return cst::fail(CSTONE_ERR_INVALID_ARG, "cstone_cube_from_bounds: bad argument");
    cst::cube_from_bounds_kernel<<<1, 32, 0, cst::as_stream(stream)>>>(bounds, box);
    CST_LAUNCHED("cube_from_bounds_kernel");
    return CSTONE_OK;
}

int cstone_decompose_workspace_size(int64_t n_leaves, int32_t n_ranks, size_t* bytes) {
    if (!bytes || n_leaves < 0 || n_leaves > CSTONE_MAX_LEAVES || n_ranks < 1 || n_ranks > cst::kMaxRanks)
        return cst::fail(CSTONE_ERR_INVALID_ARG, "cstone_decompose_workspace_size: bad argument");
    *bytes = cst::dec_layout(nullptr, n_leaves, n_ranks).bytes;
    return CSTONE_OK;
}

int cstone_decompose(const uint32_t* counts, int64_t n_leaves, int32_t n_ranks, int64_t* cuts, void* ws,
                     size_t ws_bytes, void* stream) {
    if (n_leaves < 0 || n_leaves > CSTONE_MAX_LEAVES || n_ranks < 1 || n_ranks > cst::kMaxRanks || !cuts ||
        (n_leaves > 0 && !counts))
        return cst::fail(CSTONE_ERR_INVALID_ARG, "cstone_decompose: bad argument (n_leaves=%lld, n_ranks=%d)",
                         (long long)n_leaves, n_ranks);
    cst::DecLayout l = cst::dec_layout(ws, n_leaves, n_ranks);
    if (int rc = cst::check_ws(ws, ws_bytes, l.bytes, "cstone_decompose")) return rc;
    cudaStream_t st = cst::as_stream(stream);
    CST_CUDA(cudaMemsetAsync(ws, 0, sizeof(cst::WsHeader), st));
    CST_CUDA(cudaMemsetAsync(l.total, 0, sizeof(cst::u64), st));
    CST_CUDA(cudaMemsetAsync(l.hist, 0, ((size_t)n_ranks + 1) * sizeof(cst::u32), st));
    if (l.nchunks > 0) {
        cst::dec_chunk_sum_kernel<<<(unsigned)l.nchunks, cst::kDecThreads, 0, st>>>(counts, n_leaves, l.chunk);
        CST_LAUNCHED("dec_chunk_sum_kernel");
        cst::dec_scan_kernel<<<1, 1024, 0, st>>>(l.chunk, l.nchunks, l.total);
        CST_LAUNCHED("dec_scan_kernel");
        cst::dec_hist_kernel<<<(unsigned)l.nchunks, cst::kDecThreads, 0, st>>>(counts, n_leaves, l.chunk, l.total,
                                                                               n_ranks, l.hist);
        CST_LAUNCHED("dec_hist_kernel");
    }
    cst::dec_cuts_kernel<<<1, 1024, 0, st>>>(l.hist, n_ranks, n_leaves, reinterpret_cast<long long*>(cuts));
    CST_LAUNCHED("dec_cuts_kernel");
    return CSTONE_OK;
}

}  // extern "C"
