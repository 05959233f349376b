// Allocation-free triangular solve: gblu_solve_factors_noalloc.
//
// Some callers cannot call cudaMalloc at all: a circuit simulator that runs
// inside a host process with its own fixed device-memory pool, code that
// runs while a CUDA graph is being captured into a pool it does not own, or
// embedded/safety-certified builds that forbid allocation after start-up.
// They keep the LU factors in their own device buffers and only need the
// solve.  This entry point runs sync-free row solves (one warp per row,
// ready flags) like the handle's gblu_solve, but its scratch (the intermediate vector, the ready
// flags and the work tickets) lives in one file-scope static device array
// instead of handle-owned allocations.  The paper has no counterpart; it is
// an interface convenience.
//
// Limits and sharing: n <= GBLU_NOALLOC_MAX_N; the array (8 MB + 256 B) is
// held on a device from the time this module is loaded there until the
// process exits.  Within one process all calls on a device share it, so
// calls that overlap on the GPU (different streams or host threads on the
// same device) race and must be serialized by the caller; another process
// loads its own copy of the module and so has its own array.  Every call
// looks up the array's device address (cudaGetSymbolAddress, which
// allocates nothing) with the current device, so the address stays right
// after a device reset; the first call on a device also queries occupancy,
// so make it before any stream capture.
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

#include "gblu_internal.h"

namespace {

constexpr int kMaxDevices = 64;
constexpr int kWarps = 8;
constexpr unsigned kFull = 0xffffffffu;
constexpr long long kDefaultSpinLimit = 1LL << 24;

// layout: y double[MAX_N] | lflag int32[MAX_N] | uflag int32[MAX_N] | ctl int32[64]
constexpr size_t kYBytes = (size_t)GBLU_NOALLOC_MAX_N * sizeof(double);
constexpr size_t kFlagBytes = (size_t)GBLU_NOALLOC_MAX_N * sizeof(int32_t);
constexpr size_t kCtlBytes = 256;
constexpr size_t kScratchBytes = kYBytes + 2 * kFlagBytes + kCtlBytes;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

struct Scratch {
    double *y;
    int32_t *lflag, *uflag;
    int32_t *ctl;  // [0] ticket L, [1] ticket U, [2] status
    long long spin_limit;
};

__device__ __forceinline__ int ld_acquire(const int32_t *p)
{
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release(int32_t *p, int v)
{
    asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ double warp_sum(double v)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

// the flags hold 0/1 and must start at 0 on every call: the array keeps the
// previous call's contents
__global__ void noalloc_clear_kernel(Scratch s, int n)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        s.lflag[i] = 0;
        s.uflag[i] = 0;
    }
    if (blockIdx.x == 0 && threadIdx.x < 3) s.ctl[threadIdx.x] = 0;
}

__device__ bool wait_flag(const int32_t *flag, Scratch s)
{
    long long it = 0;
    while (ld_acquire(flag) != 1) {
        // the shared status word is read only every 64 polls
        if (++it > s.spin_limit || ((it & 63) == 0 && *(volatile int32_t *)(s.ctl + 2) != 0)) {
            atomicCAS(s.ctl + 2, 0, GBLU_ERR_DEVICE_TIMEOUT);
            return false;
        }
        __nanosleep(32);
    }
    return true;
}

// y = L^-1 (P b), rows in increasing order (a topological order of L)
__global__ void __launch_bounds__(kWarps * 32)
noalloc_lsolve_kernel(int n, const int64_t *Lrp, const int32_t *Lcol, const double *Lval,
                      const int32_t *piv, const double *b, Scratch s)
{
    const int lane = threadIdx.x & 31;
    for (;;) {
        int i = 0;
        if (lane == 0) i = atomicAdd(s.ctl + 0, 1);
        i = __shfl_sync(kFull, i, 0);
        if (i >= n) break;
        double acc = 0.0;
        bool ok = true;
        for (int64_t e = Lrp[i] + lane; e < Lrp[i + 1]; e += 32) {
            const int j = Lcol[e];
            ok = ok && wait_flag(s.lflag + j, s);
            acc = fma(Lval[e], __ldcg(s.y + j), acc);
        }
        acc = warp_sum(acc);
        if (lane == 0) {
            s.y[i] = b[piv[i]] - acc;
            __threadfence();
            st_release(s.lflag + i, 1);
        }
        if (__any_sync(kFull, !ok)) break;
    }
}

// z = U^-1 y in decreasing row order, x(q) = z
__global__ void __launch_bounds__(kWarps * 32)
noalloc_usolve_kernel(int n, const int64_t *Urp, const int32_t *Ucol, const double *Uval,
                      const double *Udiag, const int32_t *q, double *x, Scratch s)
{
    const int lane = threadIdx.x & 31;
    for (;;) {
        int t = 0;
        if (lane == 0) t = atomicAdd(s.ctl + 1, 1);
        t = __shfl_sync(kFull, t, 0);
        if (t >= n) break;
        const int i = n - 1 - t;
        double acc = 0.0;
        bool ok = true;
        for (int64_t e = Urp[i] + lane; e < Urp[i + 1]; e += 32) {
            const int j = Ucol[e];
            ok = ok && wait_flag(s.uflag + j, s);
            acc = fma(Uval[e], __ldcg(s.y + j), acc);
        }
        acc = warp_sum(acc);
        if (lane == 0) {
            const double z = (__ldcg(s.y + i) - acc) / Udiag[i];
            s.y[i] = z;
            x[q[i]] = z;
            __threadfence();
            st_release(s.uflag + i, 1);
        }
        if (__any_sync(kFull, !ok)) break;
    }
}

__global__ void noalloc_status_kernel(Scratch s, int32_t *status_dev)
{
    *status_dev = s.ctl[2];
}

struct DeviceSetup {
    bool ready = false;
    int grid = 0;
};

std::mutex g_setup_mutex;
DeviceSetup g_setup[kMaxDevices];

}  // namespace

extern "C" int gblu_solve_factors_noalloc(int32_t n, const int64_t *Lrp, const int32_t *Lcol,
                                          const double *Lval, const int64_t *Urp,
                                          const int32_t *Ucol, const double *Uval,
                                          const double *Udiag, const int32_t *piv,
                                          const int32_t *q, const double *b_dev, double *x_dev,
                                          int32_t *status_dev, long long spin_limit, void *stream)
{
    using gblu::record_error;
    if (n < 1 || n > GBLU_NOALLOC_MAX_N)
        return record_error(GBLU_ERR_INVALID_INPUT,
                            "gblu_solve_factors_noalloc: n must be in [1, GBLU_NOALLOC_MAX_N = 524288]");
    if (!Lrp || !Lcol || !Lval || !Urp || !Ucol || !Uval || !Udiag || !piv || !q || !b_dev ||
        !x_dev || b_dev == x_dev)
        return record_error(GBLU_ERR_INVALID_INPUT,
                            "gblu_solve_factors_noalloc: null pointer or b_dev == x_dev");
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return record_error(GBLU_ERR_CUDA, "gblu_solve_factors_noalloc: no usable current device");
    // every call, with the device current: the host-side name of the array
    // is not a device address, and the address can change when the module
    // is loaded again after a device reset
    void *ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr) {
        cudaGetLastError();
        return record_error(GBLU_ERR_CUDA, "gblu_solve_factors_noalloc: cudaGetSymbolAddress failed");
    }
    unsigned char *base = static_cast<unsigned char *>(ptr);
    DeviceSetup *ds = &g_setup[dev];
    {
        // the grid size, once per device
        std::lock_guard<std::mutex> lock(g_setup_mutex);
        if (!ds->ready) {
            int sms = 0, per_l = 0, per_u = 0;
            if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
                cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_l, noalloc_lsolve_kernel,
                                                              kWarps * 32, 0) != cudaSuccess ||
                cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_u, noalloc_usolve_kernel,
                                                              kWarps * 32, 0) != cudaSuccess) {
                cudaGetLastError();
                return record_error(GBLU_ERR_CUDA, "gblu_solve_factors_noalloc: device query failed");
            }
            ds->grid = sms * (per_l < per_u ? per_l : per_u);
            if (ds->grid < 1) ds->grid = 1;
            ds->ready = true;
        }
    }
    Scratch s;
    s.y = reinterpret_cast<double *>(base);
    s.lflag = reinterpret_cast<int32_t *>(base + kYBytes);
    s.uflag = reinterpret_cast<int32_t *>(base + kYBytes + kFlagBytes);
    s.ctl = reinterpret_cast<int32_t *>(base + kYBytes + 2 * kFlagBytes);
    s.spin_limit = spin_limit > 0 ? spin_limit : kDefaultSpinLimit;
    cudaStream_t st = (cudaStream_t)stream;
    const int cgrid = (n + 255) / 256 < 1024 ? (n + 255) / 256 : 1024;
    noalloc_clear_kernel<<<cgrid, 256, 0, st>>>(s, n);
    noalloc_lsolve_kernel<<<ds->grid, kWarps * 32, 0, st>>>(n, Lrp, Lcol, Lval, piv, b_dev, s);
    noalloc_usolve_kernel<<<ds->grid, kWarps * 32, 0, st>>>(n, Urp, Ucol, Uval, Udiag, q, x_dev, s);
    if (status_dev) noalloc_status_kernel<<<1, 1, 0, st>>>(s, status_dev);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return record_error(GBLU_ERR_CUDA, cudaGetErrorString(e));
    return GBLU_OK;
}
