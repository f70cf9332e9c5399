// The rest of the Gibbs cycle of Sec. S1 around the beta draw: tau | beta,
// lambda; lambda | beta, tau; omega | beta ~ PolyaGamma(1, x_i^T beta); and the
// Gaussian vectors eta, delta of Prop. 2.1.  Horseshoe prior (half-Cauchy
// lambda_j and tau), updated through the auxiliary variables nu_j, xi of
// Makalic and Schmidt (2016):
//   xi ~ IG(1, 1 + 1/tau^2);  tau^2 ~ IG((p+1)/2, 1/xi + sum_j beta_j^2 / (2 lambda_j^2))
//   nu_j ~ IG(1, 1 + 1/lambda_j^2);  lambda_j^2 ~ IG(1, 1/nu_j + beta_j^2 / (2 tau^2))
// with IG(a, b) = b / Gamma(a, 1).
//
// Random numbers: Philox4x32-10 (Salmon, Moraes, Dror and Shaw 2011), keyed
// by the 64-bit seed, with the counter (element, stream, Gibbs step, block):
// every element draws from its own counter, so the result does not depend
// on how threads are scheduled.  Each block yields two uniforms in (0, 1)
// with 53 random bits; exponentials by inversion, normals by Box-Muller (the
// cosine branch), Gamma by Marsaglia and Tsang, PolyaGamma(1, c) by
// Devroye's alternating series as given by Polson, Scott and Windle (2013).
// All arithmetic is float64.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>

#include "device_common.cuh"
#include "internal.h"

namespace pcg {

enum : uint32_t {
    kStreamXi = 1, kStreamTau = 2, kStreamNu = 3, kStreamLambda = 4,
    kStreamOmega = 5, kStreamEta = 6, kStreamDelta = 7
};

constexpr double kPi = 3.141592653589793;
constexpr double kPi2 = 9.869604401089358;   // pi^2
constexpr double kTwoPi = 6.283185307179586;

// Philox4x32-10: ten rounds of two 32x32 -> 64-bit products, the key bumped
// by the Weyl increments after every round.
__device__ __forceinline__ void philox10(uint32_t &c0, uint32_t &c1, uint32_t &c2, uint32_t &c3,
                                         uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t hi0 = __umulhi(0xD2511F53u, c0), lo0 = 0xD2511F53u * c0;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c2), lo1 = 0xCD9E8D57u * c2;
        const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
}

struct Rng {
    uint32_t k0, k1, idx, stream, step, block;
    double buf[2];
    int have;
};

__device__ __forceinline__ Rng rng_at(uint64_t seed, uint32_t idx, uint32_t stream, uint32_t step) {
    Rng g;
    g.k0 = (uint32_t)seed;
    g.k1 = (uint32_t)(seed >> 32);
    g.idx = idx;
    g.stream = stream;
    g.step = step;
    g.block = 0;
    g.have = 0;
    return g;
}

__device__ __forceinline__ double u53(uint32_t a, uint32_t b) {
    return ((double)(a >> 5) * 67108864.0 + (double)(b >> 6) + 0.5) * (1.0 / 9007199254740992.0);
}

__device__ double rng_uniform(Rng &g) {
    if (g.have == 0) {
        uint32_t c0 = g.idx, c1 = g.stream, c2 = g.step, c3 = g.block;
        philox10(c0, c1, c2, c3, g.k0, g.k1);
        g.block += 1;
        g.buf[0] = u53(c0, c1);
        g.buf[1] = u53(c2, c3);
        g.have = 2;
    }
    g.have -= 1;
    return g.buf[1 - g.have];
}

__device__ __forceinline__ double rng_exp(Rng &g) { return -log(rng_uniform(g)); }

__device__ __forceinline__ double rng_normal(Rng &g) {
    const double u1 = rng_uniform(g), u2 = rng_uniform(g);
    return sqrt(-2.0 * log(u1)) * cos(kTwoPi * u2);
}

// Gamma(a, 1), a >= 1 (Marsaglia and Tsang).  The attempt cap only ends a
// broken input (NaN); a valid shape accepts within a few attempts.
__device__ double rng_gamma(Rng &g, double a) {
    const double d = a - 1.0 / 3.0, c = 1.0 / sqrt(9.0 * d);
    for (int attempt = 0; attempt < 100000; ++attempt) {
        const double x = rng_normal(g);
        double v = 1.0 + c * x;
        if (v <= 0.0) continue;
        v = v * v * v;
        const double u = rng_uniform(g);
        if (log(u) < 0.5 * x * x + d - d * v + d * log(v)) return d * v;
    }
    return nan("");
}

__device__ __forceinline__ double norm_cdf(double x) { return 0.5 * erfc(-x / 1.4142135623730951); }

// n-th term of the alternating series of the J*(1, 0) density, split at t
__device__ __forceinline__ double pg_term(int n, double x, double t) {
    const double h = n + 0.5;
    if (x > t) return kPi * h * exp(-h * h * kPi2 * x / 2.0);
    return kPi * h * pow(2.0 / (kPi * x), 1.5) * exp(-2.0 * h * h / x);
}

// IG(1/z, 1) truncated to (0, t)
__device__ double pg_trunc_ig(Rng &g, double z, double t) {
    const double mu = z > 0.0 ? 1.0 / z : INFINITY;
    if (mu > t) {
        for (int attempt = 0; attempt < 100000; ++attempt) {
            double e1, e2;
            do {
                e1 = rng_exp(g);
                e2 = rng_exp(g);
            } while (e1 * e1 > 2.0 * e2 / t);
            const double x = t / ((1.0 + t * e1) * (1.0 + t * e1));
            if (rng_uniform(g) <= exp(-0.5 * z * z * x)) return x;
        }
        return nan("");
    }
    for (int attempt = 0; attempt < 100000; ++attempt) {
        const double y0 = rng_normal(g);
        const double y = y0 * y0;
        double x = mu + 0.5 * mu * mu * y - 0.5 * mu * sqrt(4.0 * mu * y + (mu * y) * (mu * y));
        if (rng_uniform(g) > mu / (mu + x)) x = mu * mu / x;
        if (x <= t) return x;
    }
    return nan("");
}

// PolyaGamma(1, c) = J*(1, |c|/2) / 4
__device__ double pg1(double c, Rng &g) {
    const double t = 0.64, z = 0.5 * fabs(c);
    const double K = kPi2 / 8.0 + 0.5 * z * z;
    const double p = kPi / (2.0 * K) * exp(-K * t);
    double q;
    if (z > 0.0) {
        const double mu = 1.0 / z, rt = sqrt(1.0 / t);
        q = 2.0 * exp(-z) * (norm_cdf(rt * (t / mu - 1.0)) + exp(2.0 / mu) * norm_cdf(-rt * (t / mu + 1.0)));
    } else {
        q = 4.0 * norm_cdf(-sqrt(1.0 / t));
    }
    const double r = p / (p + q);
    for (int attempt = 0; attempt < 100000; ++attempt) {
        double x;
        if (rng_uniform(g) < r) x = t + rng_exp(g) / K;
        else x = pg_trunc_ig(g, z, t);
        double s = pg_term(0, x, t);
        const double y = rng_uniform(g) * s;
        for (int n = 1; n < 1000; ++n) {
            if (n & 1) {
                s -= pg_term(n, x, t);
                if (y <= s) return 0.25 * x;
            } else {
                s += pg_term(n, x, t);
                if (y > s) break;
            }
        }
    }
    return nan("");
}

// steps 1 (tau, xi): one block; sc = {tau, xi} in and out
__global__ void __launch_bounds__(1024) k_g_tau(int64_t p, const double *__restrict__ beta,
                                                const double *__restrict__ lam, double *sc, uint64_t seed,
                                                uint32_t step) {
    __shared__ double red[32];
    double acc = 0.0;
    for (int64_t j = threadIdx.x; j < p; j += blockDim.x) {
        const double b = beta[j], l = lam[j];
        acc += b * b / (2.0 * l * l);
    }
    const double ssq = block_sum(acc, red);
    if (threadIdx.x == 0) {
        const double tau = sc[0];
        Rng g = rng_at(seed, 0u, kStreamXi, step);
        const double xi = (1.0 + 1.0 / (tau * tau)) / rng_exp(g);
        Rng h = rng_at(seed, 0u, kStreamTau, step);
        sc[0] = sqrt((1.0 / xi + ssq) / rng_gamma(h, 0.5 * (double)(p + 1)));
        sc[1] = xi;
    }
}

// step 2 (nu, lambda), per coefficient, with the new tau
__global__ void __launch_bounds__(256) k_g_lambda(int64_t p, const double *__restrict__ beta, double *lam,
                                                  double *nu, const double *sc, uint64_t seed, uint32_t step) {
    const double tau = sc[0];
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < p; j += (int64_t)gridDim.x * blockDim.x) {
        const double l = lam[j], b = beta[j];
        Rng g = rng_at(seed, (uint32_t)j, kStreamNu, step);
        const double v = (1.0 + 1.0 / (l * l)) / rng_exp(g);
        Rng h = rng_at(seed, (uint32_t)j, kStreamLambda, step);
        nu[j] = v;
        lam[j] = sqrt((1.0 / v + b * b / (2.0 * tau * tau)) / rng_exp(h));
    }
}

// psi = X beta (float64 gathers, G lanes per row)
template <int G>
__global__ void __launch_bounds__(256) k_g_psi(int64_t n, const int64_t *__restrict__ row_ptr,
                                               const int32_t *__restrict__ col_idx,
                                               const double *__restrict__ beta, double *__restrict__ psi) {
    const int lane = threadIdx.x & (G - 1);
    const int64_t gpw = 32 / G;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t sub = (threadIdx.x & 31) / G;
    for (int64_t base = warp * gpw; base < n; base += nwarps * gpw) {
        const int64_t i = base + sub;
        double acc = 0.0;
        if (i < n) acc = segment_partial<G, double>(col_idx, row_ptr[i], row_ptr[i + 1], beta, lane);
        acc = group_sum<G>(acc);
        if (i < n && lane == 0) psi[i] = acc;
    }
}

// step 3 and step 4's eta: omega_i ~ PG(1, psi_i), z_i = (y_i - 1/2) / omega_i, eta_i ~ N(0, 1)
__global__ void __launch_bounds__(256) k_g_omega(int64_t n, const double *__restrict__ psi,
                                                 const double *__restrict__ y, double *__restrict__ omega,
                                                 double *__restrict__ z, double *__restrict__ eta,
                                                 uint64_t seed, uint32_t step) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        Rng g = rng_at(seed, (uint32_t)i, kStreamOmega, step);
        const double w = pg1(psi[i], g);
        omega[i] = w;
        z[i] = (y[i] - 0.5) / w;
        Rng h = rng_at(seed, (uint32_t)i, kStreamEta, step);
        eta[i] = rng_normal(h);
    }
}

// step 4's delta ~ N(0, I_p)
__global__ void __launch_bounds__(256) k_g_delta(int64_t p, double *__restrict__ delta, uint64_t seed,
                                                 uint32_t step) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < p; j += (int64_t)gridDim.x * blockDim.x) {
        Rng g = rng_at(seed, (uint32_t)j, kStreamDelta, step);
        delta[j] = rng_normal(g);
    }
}

// ===========================================================================
// host side: steps 1-3 and the Gaussian vectors; the beta draw follows in
// pcg_gibbs_step (capi.cu) through the single-RHS path
// ===========================================================================
pcg_status run_gibbs_updates(pcg_ctx *ctx, const pcg_csr *Xr, const double *y, uint64_t seed, uint32_t step,
                             double *omega, double *lambda, double *nu, double *tau, double *xi,
                             const double *beta, const double **z_out, const double **eta_out,
                             const double **delta_out) {
    const int64_t n = Xr->n, p = Xr->p;
    cudaError_t e;
    const size_t nn = (size_t)std::max<int64_t>(n, 1), np = (size_t)std::max<int64_t>(p, 1);
    double *bn = (double *)grow(ctx, "gibbs:n", sizeof(double) * 3 * nn, &e);
    double *bp = (double *)grow(ctx, "gibbs:p", sizeof(double) * np, &e);
    double *sc = (double *)grow(ctx, "gibbs:sc", sizeof(double) * 2, &e);
    double *hs = (double *)grow_host(ctx, "gibbs:hsc", sizeof(double) * 2, &e);
    if (!bn || !bp || !sc || !hs) return cuda_error(ctx, e, "allocating the Gibbs workspace");
    double *psi = bn, *z = bn + nn, *eta = bn + 2 * nn, *delta = bp;
    cudaStream_t s = ctx->stream;
    hs[0] = *tau;
    hs[1] = *xi;
    PCG_CUDA_TRY(ctx, cudaMemcpyAsync(sc, hs, sizeof(double) * 2, cudaMemcpyHostToDevice, s));
    const int grid = std::min(ctx->num_sms * 8, kMaxReduceBlocks);
    const int grid_p = (int)std::max<int64_t>(1, std::min<int64_t>((p + 255) / 256, ctx->num_sms * 8));
    const int grid_n = (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, ctx->num_sms * 8));
    PCG_PROF(ctx, "g_tau", k_g_tau<<<1, 1024, 0, s>>>(p, beta, lambda, sc, seed, step));
    PCG_PROF(ctx, "g_lambda", k_g_lambda<<<grid_p, 256, 0, s>>>(p, beta, lambda, nu, sc, seed, step));
    if (n > 0) {
        const double mean = (double)Xr->nnz / (double)n;
        const int G = mean < 6 ? 4 : mean < 20 ? 8 : mean < 56 ? 16 : 32;
        switch (G) {
            case 4: PCG_PROF(ctx, "g_psi", (k_g_psi<4><<<grid, 256, 0, s>>>(n, Xr->row_ptr, Xr->col_idx, beta, psi))); break;
            case 8: PCG_PROF(ctx, "g_psi", (k_g_psi<8><<<grid, 256, 0, s>>>(n, Xr->row_ptr, Xr->col_idx, beta, psi))); break;
            case 16: PCG_PROF(ctx, "g_psi", (k_g_psi<16><<<grid, 256, 0, s>>>(n, Xr->row_ptr, Xr->col_idx, beta, psi))); break;
            default: PCG_PROF(ctx, "g_psi", (k_g_psi<32><<<grid, 256, 0, s>>>(n, Xr->row_ptr, Xr->col_idx, beta, psi))); break;
        }
        PCG_PROF(ctx, "g_omega", k_g_omega<<<grid_n, 256, 0, s>>>(n, psi, y, omega, z, eta, seed, step));
    }
    PCG_PROF(ctx, "g_delta", k_g_delta<<<grid_p, 256, 0, s>>>(p, delta, seed, step));
    PCG_CUDA_TRY(ctx, cudaGetLastError());
    PCG_CUDA_TRY(ctx, cudaMemcpyAsync(hs, sc, sizeof(double) * 2, cudaMemcpyDeviceToHost, s));
    PCG_CUDA_TRY(ctx, cudaStreamSynchronize(s));
    prof_collect(ctx);
    *tau = hs[0];
    *xi = hs[1];
    *z_out = z;
    *eta_out = eta;
    *delta_out = delta;
    if (!(isfinite(*tau) && *tau > 0.0) || !(isfinite(*xi) && *xi > 0.0))
        return set_error(ctx, PCG_NONFINITE, "tau or xi update gave a non-finite or non-positive value");
    return PCG_OK;
}

}  // namespace pcg
