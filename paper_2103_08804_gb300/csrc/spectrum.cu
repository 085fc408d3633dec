// The spectral function on a frequency grid: the Chebyshev sum of Sec. II
// (Eq. Aw) with the Jackson damping of Sec. V, and the resolvent of the
// Krylov projection of Sec. IV at omega + i eta (its continued fraction is
// the same function written as a sum over the projected poles).
//
// Frequencies omega = E - E0 map to omega' = omega / a - W' in [-1, 1].
// One thread per frequency; the damped coefficients g_n mu_n are formed once
// per CTA in shared memory, then T_n(omega') follows the three-term
// recursion T_{n+1} = 2 x T_n - T_{n-1} (stable for |x| < 1).  float64.
#include "common.cuh"

namespace {

constexpr int SP_THREADS = 256;

__global__ void __launch_bounds__(SP_THREADS) spectrum_kernel(const double* __restrict__ mu_,
                                                              int Nm, double a, double Wp,
                                                              int jackson,
                                                              const double* __restrict__ omega,
                                                              int n_omega,
                                                              double* __restrict__ A_) {
    extern __shared__ __align__(16) unsigned char sm[];
    cpx<double>* c = (cpx<double>*)sm;  // [Nm] g_n mu_n
    const cpx<double>* mu = (const cpx<double>*)mu_;
    const double q = 3.14159265358979323846 / (Nm + 1);
    for (int n = threadIdx.x; n < Nm; n += blockDim.x) {
        double g = 1.0;
        if (jackson) {
            double s, co, s1, c1;
            sincos(q * n, &s, &co);
            sincos(q, &s1, &c1);
            g = ((Nm - n + 1) * co + s * c1 / s1) / (Nm + 1);
        }
        c[n] = g * mu[n];
    }
    __syncthreads();
    const int w = blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= n_omega) return;
    const double x = omega[w] / a - Wp;
    cpx<double> out = {0.0, 0.0};
    if (x > -1.0 && x < 1.0) {
        cpx<double> s = c[0];
        double t0 = 1.0, t1 = x;
        for (int n = 1; n < Nm; ++n) {
            s = s + (2.0 * t1) * c[n];
            const double t2 = 2.0 * x * t1 - t0;
            t0 = t1;
            t1 = t2;
        }
        out = (1.0 / (a * 3.14159265358979323846 * sqrt(1.0 - x * x))) * s;
    }
    ((cpx<double>*)A_)[w] = out;
}

// A(omega) = -Im sum_k w_k / (omega' + i eta / a - lambda_k) / (pi a)
//          = sum_k w_k (eta / a) / ((omega' - lambda_k)^2 + (eta / a)^2) / (pi a)
__global__ void __launch_bounds__(SP_THREADS) lorentzian_kernel(const double* __restrict__ poles,
                                                                const double* __restrict__ weights,
                                                                int K, double a, double Wp,
                                                                double eta,
                                                                const double* __restrict__ omega,
                                                                int n_omega,
                                                                double* __restrict__ A) {
    const int w = blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= n_omega) return;
    const double x = omega[w] / a - Wp, e = eta / a;
    double s = 0.0;
    for (int k = 0; k < K; ++k) {
        const double d = x - poles[k];
        s += weights[k] * e / (d * d + e * e);
    }
    A[w] = s / (3.14159265358979323846 * a);
}

}  // namespace

extern "C" cr_status cheb_spectrum(cr_ctx* ctx, const double* mu, int Nm, double a, double Wp,
                                   int jackson, const double* omega, int n_omega,
                                   double* A_out) {
    if (!ctx) return CR_EINVAL;
    CR_CHECK_ARG(Nm >= 1 && (size_t)Nm * 16 <= 200 * 1024, "cheb_spectrum: Nm=%d outside [1, 12800]", Nm);
    CR_CHECK_ARG(n_omega >= 0, "cheb_spectrum: n_omega < 0");
    CR_CHECK_ARG(a > 0.0 && Wp > 0.0 && Wp < 1.0, "cheb_spectrum: need a > 0 and 0 < W' < 1");
    CR_CHECK_ARG(jackson == 0 || jackson == 1, "cheb_spectrum: jackson must be 0 or 1");
    if (n_omega == 0) return CR_OK;
    CR_CHECK_ARG(mu && omega && A_out, "cheb_spectrum: null array");
    const size_t sm = (size_t)Nm * 16;
    if (sm > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(spectrum_kernel,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return cr_fail(ctx, CR_ECUDA, "cheb_spectrum: %s", cudaGetErrorString(e));
    }
    CR_LAUNCH(ctx, CR_K_OTHER,
              spectrum_kernel<<<(n_omega + SP_THREADS - 1) / SP_THREADS, SP_THREADS, sm,
                                ctx->stream>>>(mu, Nm, a, Wp, jackson, omega, n_omega, A_out));
    return cr_check_launch(ctx, "spectrum_kernel");
}

extern "C" cr_status cheb_lorentzian(cr_ctx* ctx, const double* poles, const double* weights,
                                     int K, double a, double Wp, double eta,
                                     const double* omega, int n_omega, double* A_out) {
    if (!ctx) return CR_EINVAL;
    CR_CHECK_ARG(K >= 0 && n_omega >= 0, "cheb_lorentzian: negative size");
    CR_CHECK_ARG(a > 0.0 && eta > 0.0, "cheb_lorentzian: need a > 0 and eta > 0");
    if (n_omega == 0) return CR_OK;
    CR_CHECK_ARG(omega && A_out && (K == 0 || (poles && weights)), "cheb_lorentzian: null array");
    CR_LAUNCH(ctx, CR_K_OTHER,
              lorentzian_kernel<<<(n_omega + SP_THREADS - 1) / SP_THREADS, SP_THREADS, 0,
                                  ctx->stream>>>(poles, weights, K, a, Wp, eta, omega, n_omega,
                                                 A_out));
    return cr_check_launch(ctx, "lorentzian_kernel");
}
