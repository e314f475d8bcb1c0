// Internal helpers of the cstone library: status handling, workspace carving, bounded waits.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

#include "cstone.h"

// Key length of this build. Every translation unit that depends on it is compiled twice: by
// default for 63-bit keys (L = 21, uint64 words, namespace cst, entry points cstone_*), and with
// CSTONE_KEY32 for 30-bit keys (L = 10, uint32 words, namespace cst30, entry points cstone30_*),
// the two key lengths Sec. 3 names. Status handling, workspace carving and device helpers below
// are shared by both.
#define CST_STR2(x) #x
#define CST_STR(x) CST_STR2(x)  // CST_STR(CSTONE_FN(sort)) is the entry point's name as a string

#ifdef CSTONE_KEY32
#define CST_NS cst30
#define CSTONE_FN(name) cstone30_##name
#define CST_KEY_C uint32_t  // key word in the C signatures
#else
#define CST_NS cst
#define CSTONE_FN(name) cstone_##name
#define CST_KEY_C uint64_t
#endif

namespace cst {

using u64 = unsigned long long;
using u32 = unsigned int;

// ---------------------------------------------------------------- host-side status plumbing
int fail(int status, const char* fmt, ...);
int cuda_fail(cudaError_t e, const char* what);
int sm_count();
void note_launch();  // counts a kernel launch of this library (cstone_kernel_launches)

#define CST_CUDA(call)                                          \
    do {                                                        \
        cudaError_t cst_e_ = (call);                            \
        if (cst_e_ != cudaSuccess) return cst::cuda_fail(cst_e_, #call); \
    } while (0)

#define CST_LAUNCHED(name)              \
    do {                                \
        cst::note_launch();             \
        CST_CUDA(cudaGetLastError());   \
    } while (0)

// A cooperative launch: counted, then checked like any CUDA call.
#define CST_COOP(call)        \
    do {                      \
        cst::note_launch();   \
        CST_CUDA(call);       \
    } while (0)

inline cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

// Every workspace starts with this header; err is the device error word of the call.
struct WsHeader {
    u32 err;        // 0 = ok, else a cstone_status (TIMEOUT, CAPACITY, ...)
    u32 err_info;   // free-form detail (e.g. where a wait gave up)
    u32 pad[62];
};
static_assert(sizeof(WsHeader) == 256, "header is one 256-byte slot");

// Sequential carving of a workspace into 256-byte aligned arrays. With base == nullptr it only
// measures, so the same code serves the size query and the call.
struct Carver {
    char* base;
    size_t off;
    explicit Carver(void* b) : base(static_cast<char*>(b)), off(sizeof(WsHeader)) {}
    template <class T>
    T* take(size_t count) {
        size_t bytes = ((count * sizeof(T) + 255) / 256) * 256;
        T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
        off += bytes;
        return p;
    }
    size_t size() const { return off; }
};

inline bool aligned256(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 255u) == 0; }

int check_ws(void* ws, size_t have, size_t need, const char* who);

// ---------------------------------------------------------------- device helpers
constexpr long long kSpinLimit = 1ll << 24;  // polls before a wait is declared timed out

__device__ __forceinline__ u32 ld_volatile(const u32* p) { return *reinterpret_cast<const volatile u32*>(p); }
__device__ __forceinline__ void st_volatile(u32* p, u32 v) { *reinterpret_cast<volatile u32*>(p) = v; }

__device__ __forceinline__ u32 lanemask_lt() {
    u32 m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Records the first error of a call (later ones keep the first).
__device__ __forceinline__ void raise_error(WsHeader* h, u32 status, u32 info) {
    if (atomicCAS(&h->err, 0u, status) == 0u) h->err_info = info;
}

// Grid-wide barrier for cooperative launches (all blocks co-resident). The counter only grows
// (it is zeroed before every launch): block b arrives with one release add, and round r of the
// barrier is complete once the counter reaches r * gridDim.x, which the arriving block reads off
// the value it added to. One atomic per block and no reset step (a probe of 608 blocks of 256
// threads measured 3.3 us per barrier against 4.1 us with a counter reset by the last arrival and
// a generation word). The wait is bounded: after kSpinLimit polls it records CSTONE_ERR_TIMEOUT and
// lets the block go on.
struct GridBarrier {
    u32 count;
    u32 pad;
};

__device__ __forceinline__ u32 ld_acquire_gpu(const u32* p) {
    u32 v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ inline void grid_barrier(GridBarrier* bar, WsHeader* hdr) {
    __syncthreads();
    if (threadIdx.x == 0) {
        u32 old;
        asm volatile("atom.add.release.gpu.global.u32 %0, [%1], 1;" : "=r"(old) : "l"(&bar->count) : "memory");
        const u32 target = (old / gridDim.x + 1u) * gridDim.x;
        long long polls = 0;
        while (static_cast<int>(ld_acquire_gpu(&bar->count) - target) < 0) {
            if (++polls > kSpinLimit) {
                raise_error(hdr, CSTONE_ERR_TIMEOUT, 0x1000u);
                break;
            }
        }
    }
    __syncthreads();
}

// Blocks of `threads` threads that fit on the device at once for `kernel` (cooperative grid size),
// capped at `cap_per_sm` per SM.
int cooperative_grid(const void* kernel, int threads, size_t smem, int cap_per_sm);

}  // namespace cst

namespace CST_NS {
using namespace cst;

#ifdef CSTONE_KEY32
using Key = unsigned int;  // key word
constexpr int kLevels = CSTONE30_LEVELS;  // L
#else
using Key = unsigned long long;
constexpr int kLevels = CSTONE_LEVELS;
#endif
constexpr int kKeyBits = 3 * kLevels;                     // bits of a key
constexpr int kWordBits = 8 * static_cast<int>(sizeof(Key));
constexpr Key kKeyEnd = static_cast<Key>(1) << kKeyBits;  // 8^L
static_assert(kKeyBits < kWordBits, "8^L must fit the key word");

// Inverse of the Hilbert state machine of the key kernels, one level at a time: entry
// state * 8 + digit = octant (x << 2 | y << 1 | z of the cell bits at that level) | next state << 3.
constexpr int kHilbertStates = 48;
struct HilbertDecodeTable {
    unsigned short one[kHilbertStates * 8];
};
const HilbertDecodeTable& hilbert_decode_table();  // built once on the host (keys.cu)

// Index (from 0) of the lowest set bit of a non-zero key, and leading zero bits of a key word.
__device__ __forceinline__ int key_ffs(Key k) {
    return sizeof(Key) == 8 ? __ffsll(static_cast<long long>(k)) - 1 : __ffs(static_cast<int>(k)) - 1;
}
__device__ __forceinline__ int key_clz(Key k) {
    return sizeof(Key) == 8 ? __clzll(static_cast<long long>(k)) : __clz(static_cast<int>(k));
}
}  // namespace CST_NS
