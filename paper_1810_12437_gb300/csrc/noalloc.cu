// pcg_phi_mul_noalloc: the product out = X^T (Omega (X v)) + tau^-2 Lambda^-2 v
// for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc: code that runs while a stream is
// being captured into a CUDA graph (an allocation there is not allowed or
// breaks the capture), host runtimes whose allocator owns all of the
// device's memory and forbids side allocations, and latency-critical loops
// where an allocation could synchronise the device.  They still pass their
// own inputs and outputs; the one intermediate this product needs, the
// length-n vector u = Omega (X v) handed from the CSR pass to the CSC pass,
// lives instead in a file-scope device array of fixed size (below).  Every
// GPU that loads the library holds that array until the process exits.
//
// Everything here is in float64, like pcg_phi_mul in PCG_PREC_FP64 mode.
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "../../include/pcg_beta.h"
#include "device_common.cuh"

namespace pcg {
namespace {

// Scratch for u (PCG_NOALLOC_MAX_N doubles = 8 MiB).  Shared by every call on
// a device; each call writes all n entries it later reads, so nothing has to
// be cleared between calls.
static __device__ __align__(256) double g_noalloc_u[PCG_NOALLOC_MAX_N];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
double *g_u_addr[kMaxDevices] = {nullptr};

// Device address of the scratch array for the current device, looked up once
// per device (the array's name in host code is only a stand-in for it).
cudaError_t scratch_address(double **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_u_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_u);
        if (e != cudaSuccess) return e;
        g_u_addr[dev] = static_cast<double *>(p);
    }
    *out = g_u_addr[dev];
    return cudaSuccess;
}

template <int G>
__global__ void __launch_bounds__(256) k_na_csr(int64_t n, const int64_t *__restrict__ rp,
                                                const int32_t *__restrict__ ci,
                                                const double *__restrict__ v,
                                                const double *__restrict__ omega,
                                                double *__restrict__ u) {
    const int lane = threadIdx.x & (G - 1);
    const int64_t gpw = 32 / G;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t sub = (threadIdx.x & 31) / G;
    for (int64_t base = warp * gpw; base < n; base += nwarps * gpw) {
        const int64_t i = base + sub;
        double acc = 0.0;
        if (i < n)
            for (int64_t k = rp[i] + lane; k < rp[i + 1]; k += G) acc += __ldg(v + __ldcs(ci + k));
        acc = group_sum<G>(acc);
        if (i < n && lane == 0) u[i] = omega[i] * acc;
    }
}

template <int G>
__global__ void __launch_bounds__(256) k_na_csc(int64_t p, const int64_t *__restrict__ cp,
                                                const int32_t *__restrict__ ri,
                                                const double *__restrict__ u,
                                                const double *__restrict__ v,
                                                const double *__restrict__ lambda, double tau,
                                                double *__restrict__ out) {
    const int lane = threadIdx.x & (G - 1);
    const int64_t gpw = 32 / G;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t sub = (threadIdx.x & 31) / G;
    for (int64_t base = warp * gpw; base < p; base += nwarps * gpw) {
        const int64_t j = base + sub;
        double acc = 0.0;
        if (j < p)
            for (int64_t k = cp[j] + lane; k < cp[j + 1]; k += G) acc += __ldg(u + __ldcs(ri + k));
        acc = group_sum<G>(acc);
        if (j < p && lane == 0) out[j] = acc + prior_prec(tau, lambda[j]) * v[j];
    }
}

int pick(double mean) { return mean < 6 ? 4 : mean < 20 ? 8 : mean < 56 ? 16 : 32; }

}  // namespace
}  // namespace pcg

extern "C" pcg_status pcg_phi_mul_noalloc(const pcg_csr *X_csr, const pcg_csc *X_csc,
                                          const double *omega, const double *lambda, double tau,
                                          const double *v, double *out, void *stream) {
    using namespace pcg;
    if (!X_csr || !X_csc) return PCG_BADARG;
    const int64_t n = X_csr->n, p = X_csr->p, nnz = X_csr->nnz;
    if (n < 0 || p < 0 || nnz < 0 || X_csc->n != n || X_csc->p != p || X_csc->nnz != nnz)
        return PCG_BADARG;
    if (n > PCG_NOALLOC_MAX_N) return PCG_BADARG;   // the scratch holds at most this many rows
    if (!(tau > 0.0)) return PCG_BADARG;
    if (p == 0) return PCG_OK;
    if ((n > 0 && (!X_csr->row_ptr || !omega)) || !X_csc->col_ptr || !lambda || !v || !out ||
        (nnz > 0 && (!X_csr->col_idx || !X_csc->row_idx)))
        return PCG_BADARG;
    double *u = nullptr;
    cudaError_t e = scratch_address(&u);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return PCG_CUDA;
    }
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return PCG_CUDA;
    }
    cudaStream_t s = (cudaStream_t)stream;
    const int grid = sms * 8;
    const int gr = pick(n > 0 ? (double)nnz / n : 1.0), gc = pick((double)nnz / p);
    if (n > 0) {
        switch (gr) {
            case 4: k_na_csr<4><<<grid, 256, 0, s>>>(n, X_csr->row_ptr, X_csr->col_idx, v, omega, u); break;
            case 8: k_na_csr<8><<<grid, 256, 0, s>>>(n, X_csr->row_ptr, X_csr->col_idx, v, omega, u); break;
            case 16: k_na_csr<16><<<grid, 256, 0, s>>>(n, X_csr->row_ptr, X_csr->col_idx, v, omega, u); break;
            default: k_na_csr<32><<<grid, 256, 0, s>>>(n, X_csr->row_ptr, X_csr->col_idx, v, omega, u); break;
        }
    }
    switch (gc) {
        case 4: k_na_csc<4><<<grid, 256, 0, s>>>(p, X_csc->col_ptr, X_csc->row_idx, u, v, lambda, tau, out); break;
        case 8: k_na_csc<8><<<grid, 256, 0, s>>>(p, X_csc->col_ptr, X_csc->row_idx, u, v, lambda, tau, out); break;
        case 16: k_na_csc<16><<<grid, 256, 0, s>>>(p, X_csc->col_ptr, X_csc->row_idx, u, v, lambda, tau, out); break;
        default: k_na_csc<32><<<grid, 256, 0, s>>>(p, X_csc->col_ptr, X_csc->row_idx, u, v, lambda, tau, out); break;
    }
    e = cudaGetLastError();
    return e == cudaSuccess ? PCG_OK : PCG_CUDA;
}
