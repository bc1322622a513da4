// noalloc.cu -- <phi|psi> for callers that cannot allocate GPU memory.
//
// mps_inner needs scratch for its float64 transfer matrices; it gets it from
// the caller's allocator (or cudaMallocAsync).  Some callers cannot allocate
// at all: code running inside another framework's memory pool that forbids
// foreign allocations, real-time loops that must not touch the allocator, or
// embedders whose budget is fixed up front.  mps_inner_noalloc computes the
// same inner product with its scratch in one file-scope device array of fixed
// size.  With lazy module loading (the CUDA default) the array is reserved on
// a device when this module is first used there, and it stays reserved on
// that device until the process exits.  The call itself allocates nothing: no
// cudaMalloc/cudaFree and no allocating routine.
//
// The result is read back with a device-to-host copy into a pageable host
// pointer and a stream synchronisation, neither of which is legal while a
// stream is being captured into a CUDA graph: a call made on a capturing
// stream is refused before anything is enqueued.
//
// The array's host-side name is only a stand-in for the symbol, not a device
// address: the device address is obtained once per device with
// cudaGetSymbolAddress (the first call on a device does this, with that device
// current) and passed to the kernels.  All calls share the array and it keeps
// the previous call's contents; the kernels below initialise what they read.
// Calls whose work overlaps on the GPU (different streams, no ordering) race
// on the array.
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>
#include <string>

#include "../../include/thc.h"
#include "common.cuh"
#include "gemm.cuh"

// 16 MiB: float64 E (chi_phi x chi_psi) and F (chi_phi x 4 chi_psi) for bonds
// up to 512 x 512 (5 * 512 * 512 * 8 bytes = 10 MiB), plus the result.
#define THC_NOALLOC_SCRATCH_BYTES (16u << 20)

static __device__ __align__(256) unsigned char g_noalloc_scratch[THC_NOALLOC_SCRATCH_BYTES];

namespace thc {
void set_last_error(const std::string& msg);  // abi.cu: message for thc_last_error()
}

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_dev[kMaxDevices] = {nullptr};

struct ErrSink {  // g_noalloc_err = "..." forwards to thc_last_error()
    ErrSink& operator=(const std::string& m) {
        thc::set_last_error(m);
        return *this;
    }
} g_noalloc_err;

struct EnvA {  // E(m, k), float64 row-major
    const double* E;
    int ld;
    __device__ __forceinline__ double operator()(int, int m, int k) const { return E[(long)m * ld + k]; }
};
template <class T>
struct SiteRowB {  // site[k*ld + n] as float64
    const T* s;
    int ld;
    __device__ __forceinline__ double operator()(int, int k, int n) const { return double(s[(long)k * ld + n]); }
};
template <class T>
struct SiteColA {  // site[k*ld + m] (transposed access)
    const T* s;
    int ld;
    __device__ __forceinline__ double operator()(int, int m, int k) const { return double(s[(long)k * ld + m]); }
};
struct EnvStore {
    double* E;
    int ld;
    __device__ __forceinline__ void operator()(int, int m, int n, double v) const { E[(long)m * ld + n] = v; }
};

__global__ void k_noalloc_start(double* E) {
    if (threadIdx.x == 0 && blockIdx.x == 0) E[0] = 1.0;  // E_0 = [1]
}

// device address of the scratch array on the current device (set up once)
thc_status scratch_address(void** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        g_noalloc_err = std::string("cudaGetDevice: ") + cudaGetErrorString(e);
        return THC_ECUDA;
    }
    if (dev < 0 || dev >= kMaxDevices) {
        g_noalloc_err = "device index out of range";
        return THC_EUNSUPPORTED;
    }
    std::lock_guard<std::mutex> g(g_mu);
    if (!g_scratch_dev[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            g_noalloc_err = std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e);
            return THC_ECUDA;
        }
        g_scratch_dev[dev] = p;
    }
    *out = g_scratch_dev[dev];
    return THC_OK;
}

template <class T>
thc_status run(const thc_mps* phi, const thc_mps* psi, double* out, cudaStream_t st, double* E, double* F,
               double* res) {
    const int L = phi->L;
    cudaError_t e;
    k_noalloc_start<<<1, 32, 0, st>>>(E);
    if ((e = cudaGetLastError()) != cudaSuccess) goto fail;
    for (int s = 0; s < L; ++s) {
        const int al = phi->bond[s], ar = phi->bond[s + 1], bl = psi->bond[s], br = psi->bond[s + 1];
        // F = E B_s : [al x bl] x [bl x 4 br]
        e = thc::launch_gemm<double>(1, al, 4 * br, bl, EnvA{E, bl}, SiteRowB<T>{(const T*)psi->site[s], 4 * br},
                                     EnvStore{F, 4 * br}, st);
        if (e != cudaSuccess) goto fail;
        // E' = A_s^T F : [(al,4) x ar]^T x [(al,4) x br]
        e = thc::launch_gemm<double>(1, ar, br, 4 * al, SiteColA<T>{(const T*)phi->site[s], ar}, EnvA{F, br},
                                     EnvStore{E, br}, st);
        if (e != cudaSuccess) goto fail;
    }
    if ((e = cudaMemcpyAsync(res, E, sizeof(double), cudaMemcpyDeviceToDevice, st)) != cudaSuccess) goto fail;
    if ((e = cudaMemcpyAsync(out, res, sizeof(double), cudaMemcpyDeviceToHost, st)) != cudaSuccess) goto fail;
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) goto fail;
    return THC_OK;
fail:
    g_noalloc_err = std::string("CUDA: ") + cudaGetErrorString(e);
    return THC_ECUDA;
}

}  // namespace

extern "C" thc_status mps_inner_noalloc(const thc_mps* phi, const thc_mps* psi, double* out_re, void* stream) {
    if (!phi || !psi || !out_re) {
        g_noalloc_err = "null argument";
        return THC_EINVAL;
    }
    // the same input limits as mps_inner
    if (phi->L != psi->L || phi->L < 2 || phi->L > THC_MAX_SITES || phi->d != 4 || psi->d != 4 ||
        phi->dtype != psi->dtype || (phi->dtype != THC_F64 && phi->dtype != THC_F32)) {
        g_noalloc_err = "phi and psi must be real (F64 or F32) MPS of equal length L in [2, 64] with d = 4";
        return THC_EINVAL;
    }
    if (phi->bond[0] != 1 || psi->bond[0] != 1 || phi->bond[phi->L] != 1 || psi->bond[psi->L] != 1) {
        g_noalloc_err = "boundary bonds must be 1";
        return THC_EINVAL;
    }
    int ma = 1, mb = 1;
    for (int b = 0; b <= phi->L; ++b) {
        if (phi->bond[b] < 1 || psi->bond[b] < 1 || phi->bond[b] > 4096 || psi->bond[b] > 4096) {
            g_noalloc_err = "bond dimensions must be in [1, 4096]";
            return THC_EINVAL;
        }
        ma = phi->bond[b] > ma ? phi->bond[b] : ma;
        mb = psi->bond[b] > mb ? psi->bond[b] : mb;
    }
    for (int s = 0; s < phi->L; ++s)
        if (!phi->site[s] || !psi->site[s]) {
            g_noalloc_err = "null site pointer";
            return THC_EINVAL;
        }
    // scratch layout: E [ma x mb], F [ma x 4 mb], result [1] (all float64, 256-byte aligned)
    auto up = [](size_t x) { return (x + 31) / 32 * 32; };
    const size_t nE = up((size_t)ma * mb), nF = up((size_t)ma * 4 * mb);
    const size_t need = (nE + nF + 32) * sizeof(double);
    if (need > THC_NOALLOC_SCRATCH_BYTES) {
        g_noalloc_err = "bond dimensions too large for the " + std::to_string(THC_NOALLOC_SCRATCH_BYTES >> 20) +
                        " MiB scratch: needs " + std::to_string(need) + " bytes (max chi_phi*chi_psi ~ 400000)";
        return THC_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        const cudaError_t e = cudaStreamIsCapturing(s, &cs);
        if (e != cudaSuccess) {
            cudaGetLastError();
            g_noalloc_err = std::string("cudaStreamIsCapturing: ") + cudaGetErrorString(e);
            return THC_ECUDA;
        }
        if (cs != cudaStreamCaptureStatusNone) {
            g_noalloc_err = "mps_inner_noalloc cannot run on a stream that is being captured";
            return THC_EUNSUPPORTED;
        }
    }
    void* base = nullptr;
    thc_status st = scratch_address(&base);
    if (st != THC_OK) return st;
    double* E = static_cast<double*>(base);
    double* F = E + nE;
    double* res = F + nF;
    if (phi->dtype == THC_F64) return run<double>(phi, psi, out_re, s, E, F, res);
    return run<float>(phi, psi, out_re, s, E, F, res);
}
