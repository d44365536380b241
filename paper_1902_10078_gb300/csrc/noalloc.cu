// Allocation-free precision solve: x = (L L^T)^{-1} b for one instance, with
// the intermediate y = L^{-1} b kept in a fixed, file-scope device array.
//
// For callers that cannot allocate device memory at all (no cudaMalloc, no
// caching allocator, no workspace they could hand over): for example code
// running inside a framework callback that forbids allocation, or a process
// whose device memory is fully reserved up front by another component.  They
// pass only the inputs and the output; every other byte this call touches is
// the static array below, which every GPU that loads the library holds until
// the process exits.
#include <mutex>

#include "sweep_launch.cuh"

namespace {

// Maximum scratch: one vector y of n elements.  16 MiB -> n <= 4,194,304 in
// FP32 or n <= 2,097,152 in FP64.
constexpr size_t kNoAllocScratchBytes = size_t(16) << 20;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// Device address of g_noalloc_scratch, looked up once per device (in host code
// the symbol itself is only a host-side stand-in, not a device address).  The
// address stays valid for the life of the device's primary context; after a
// cudaDeviceReset the library must be reloaded (the cached address is stale).
constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
void *g_scratch_ptr[kMaxDevices] = {};

bnd_status scratch_address(void **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return BND_ECUDA;
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return BND_ECUDA;
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return BND_OK;
}

}  // namespace

namespace bnd {

// One instance, one right-hand side, one thread: the forward sweep writes
// y = L^{-1} b into the scratch, the backward sweep reads it and writes x.
template <typename T, int L, bool FWD>
__global__ void noalloc_solve_kernel(int64_t n, int32_t l, const T *Lm, int64_t ld, const T *in, T *out) {
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    PlanDev P{};
    P.k = 1;
    SweepArgs<T> A{};
    A.Lin = Lm;
    A.Bin = in;
    A.Xout = out;
    A.rhs0 = 0;
    A.kk = 1;
    ChainCtx c{};
    c.n = n; c.band = 0; c.ld = ld; c.rhs = 0; c.ldr = n; c.cs = 1; c.l = l;
    c.a = 0; c.b = n; c.gseg = 0; c.warm = 0; c.inst = 0;
    c.first = true; c.last = true;
    if constexpr (L >= 1) {
        const ChainPtrs<T> ptrs = chain_ptrs(A, c);
        DirectIO<T, typename SweepOf<T, L, 1, FWD ? F_SOLVE : B_SOLVE, FWD>::type> io(ptrs);
        run_reg<T, L, 1, FWD ? F_SOLVE : B_SOLVE, FWD>(P, A, c, RUN_COLD, nullptr, io);
    } else {
        if constexpr (FWD) run_fwd_generic<T, F_SOLVE>(P, A, c);
        else run_bwd_generic<T, B_SOLVE>(P, A, c);
    }
}

template <typename T, bool FWD>
static cudaError_t launch_noalloc(int64_t n, int32_t l, const T *Lm, int64_t ld, const T *in, T *out,
                                  cudaStream_t s) {
#define BND_NA(LV) \
    case LV: noalloc_solve_kernel<T, LV, FWD><<<1, 1, 0, s>>>(n, l, Lm, ld, in, out); break;
    switch (l) {
        BND_NA(1) BND_NA(2) BND_NA(3) BND_NA(4) BND_NA(5) BND_NA(6) BND_NA(7) BND_NA(8)
        default: noalloc_solve_kernel<T, 0, FWD><<<1, 1, 0, s>>>(n, l, Lm, ld, in, out);
    }
#undef BND_NA
    return cudaGetLastError();
}

template <typename T>
static bnd_status noalloc_solve_t(int64_t n, int32_t l, const void *Lm, int64_t ld, const void *b, void *x,
                                  cudaStream_t s) {
    if ((size_t)n * sizeof(T) > kNoAllocScratchBytes) return BND_EINVAL;
    void *y = nullptr;
    const bnd_status st = scratch_address(&y);
    if (st != BND_OK) return st;
    // y is written in full by the forward sweep before the backward sweep reads it:
    // nothing in the scratch has to start at zero.
    if (launch_noalloc<T, true>(n, l, (const T *)Lm, ld, (const T *)b, (T *)y, s) != cudaSuccess) return BND_ECUDA;
    if (launch_noalloc<T, false>(n, l, (const T *)Lm, ld, (const T *)y, (T *)x, s) != cudaSuccess) return BND_ECUDA;
    return BND_OK;
}

}  // namespace bnd

namespace {
// Byte ranges [p, p + bytes) that share at least one byte.
bool overlap(const void *p, size_t pb, const void *q, size_t qb) {
    const uintptr_t a = (uintptr_t)p, c = (uintptr_t)q;
    return a < c + qb && c < a + pb;
}
}  // namespace

extern "C" bnd_status banded_solve_precision_noalloc(bnd_dtype dtype, int64_t n, int32_t l, const void *L, int64_t ld,
                                                     const void *b, void *x, void *stream) {
    if (dtype != BND_F32 && dtype != BND_F64) return BND_EINVAL;
    if (n < 1 || l < 0 || l > 1024 || ld < n || !L || !b || !x) return BND_EINVAL;
    const size_t esz = dtype == BND_F32 ? 4 : 8;
    if (((uintptr_t)L % esz) || ((uintptr_t)b % esz) || ((uintptr_t)x % esz)) return BND_EALIGN;
    // x is written while b and L are still being read: it may share no byte with either
    // (b and L may overlap each other: both are only read)
    const size_t vec_bytes = (size_t)n * esz, band_bytes = ((size_t)l * (size_t)ld + (size_t)n) * esz;
    if (overlap(x, vec_bytes, b, vec_bytes) || overlap(x, vec_bytes, L, band_bytes)) return BND_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    return dtype == BND_F32 ? bnd::noalloc_solve_t<float>(n, l, L, ld, b, x, s)
                            : bnd::noalloc_solve_t<double>(n, l, L, ld, b, x, s);
}
