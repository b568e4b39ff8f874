// Host FP64 pieces of the TBPM path: the Bessel coefficient table of the
// Chebyshev expansion (Sec. 2.2) and the windowed Fourier transform of the
// correlation into the DOS (Sec. 2.4, Eq. dos_tbpm).
#include <math.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <complex>
#include <vector>

#include "tbpm_internal.cuh"

namespace tbpm {

// J_m(z), m = 0 .. n-1, by Miller's backward recurrence
//   j_{k-1} = (2k / z) j_k - j_{k+1}
// started far above the wanted orders from (0, tiny), then normalised with
// the sum rule J_0 + 2 sum_{k>=1} J_{2k} = 1 (the generating function at
// t = 1).  Backward recurrence is the stable direction for k > z.
static void miller(double z, int n, double *J)
{
    int top = n + 30 + (int)sqrt(40.0 * (n + z));
    if (top % 2) ++top;
    std::vector<double> j(top + 2, 0.0);
    j[top + 1] = 0.0;
    j[top] = 1e-300;
    double inv_z = 1.0 / z;
    for (int k = top; k >= 1; --k) {
        j[k - 1] = 2.0 * k * inv_z * j[k] - j[k + 1];
        if (fabs(j[k - 1]) > 1e250) {          // rescale to stay finite
            for (int q = k - 1; q <= top + 1; ++q) j[q] *= 1e-250;
        }
    }
    double norm = j[0];
    for (int k = 2; k <= top; k += 2) norm += 2.0 * j[k];
    for (int m = 0; m < n; ++m) J[m] = j[m] / norm;
}

int bessel_miller(double z, double tol, int max_terms, double *J, int *n_terms)
{
    if (!(z > 0.0) || z > 1000.0 || !(tol > 0.0) || max_terms < 2 || !J || !n_terms)
        return TBPM_E_INVALID_ARG;
    int want = (int)z + 80 > max_terms ? (int)z + 80 : max_terms;
    std::vector<double> all(want + 1);
    miller(z, want + 1, all.data());
    int M = -1;
    for (int m = 0; m <= want; ++m) {
        if ((double)m > z && fabs(all[m]) < tol) { M = m; break; }
    }
    if (M < 0 || M > max_terms) return TBPM_E_UNSUPPORTED;
    for (int m = 0; m < max_terms; ++m) J[m] = m < M ? all[m] : 0.0;
    *n_terms = M;
    return TBPM_OK;
}

// Adjoint of the DOS transform: for dL/dD_k on the bin centres, the
// derivative of L with respect to the averaged correlation,
//   gbar_n = dL/dRe C_n + i dL/dIm C_n,
//   gbar_0 = (tau / 2 pi) sum_k dL/dD_k,
//   gbar_n = (tau / pi) w_n sum_k dL/dD_k exp(-i E_k n tau),  0 < n < N,
//   gbar_N = 0.
// The phase exp(-i E_k n tau) advances by one rotation per n and is
// re-anchored from cos/sin every 64 steps.
// In-place radix-2 complex FFT, X_k = sum_n x_n e^{-2 pi i n k / N}, N a power
// of two (iterative Cooley-Tukey: bit reversal, then butterflies).
static void fft(std::vector<std::complex<double>> &x)
{
    const size_t n = x.size();
    for (size_t i = 1, j = 0; i < n; ++i) {
        size_t bit = n >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) std::swap(x[i], x[j]);
    }
    for (size_t len = 2; len <= n; len <<= 1) {
        const double ang = -2.0 * M_PI / (double)len;
        for (size_t i = 0; i < n; i += len)
            for (size_t k = 0; k < len / 2; ++k) {
                const std::complex<double> w(cos(ang * (double)k), sin(ang * (double)k));
                const std::complex<double> u = x[i + k], v = x[i + k + len / 2] * w;
                x[i + k] = u + v;
                x[i + k + len / 2] = u - v;
            }
    }
}

// Fermi function on the rescaled axis, 1 / (e^{b (x - m)} + 1), without overflow.
static double fermi(double x, double b, double m)
{
    const double a = b * (x - m);
    if (a > 0.0) {
        const double e = exp(-a);
        return e / (1.0 + e);
    }
    return 1.0 / (1.0 + exp(a));
}

// c_k = (2/N) sum_n f(cos(2 pi n / N)) cos(2 pi n k / N): the trapezoid rule of
// c_k = (2/pi) int_0^pi f(cos t) cos(k t) dt, by FFT (Sec. 2.2).  N doubles
// until it is at least 4 (K + 1) for the K kept terms (|c_k| > tol max|c|).
int fermi_coefficients(double beta_s, double mu_s, double tol, int k_max, std::vector<double> &c)
{
    if (!(beta_s > 0.0) || !std::isfinite(beta_s) || !std::isfinite(mu_s) || !(tol > 0.0) ||
        k_max < 1)
        return TBPM_E_INVALID_ARG;
    for (size_t n = 1024;; n *= 2) {
        std::vector<std::complex<double>> x(n);
        for (size_t i = 0; i < n; ++i)
            x[i] = fermi(cos(2.0 * M_PI * (double)i / (double)n), beta_s, mu_s);
        fft(x);
        double cmax = 0.0;
        for (size_t k = 0; k < n / 2; ++k) cmax = std::max(cmax, fabs(x[k].real()));
        size_t K = 1;
        for (size_t k = 0; k < n / 2; ++k)
            if (fabs(x[k].real()) > tol * cmax) K = k + 1;
        if (4 * (K + 1) <= n || n >= (size_t)16 * k_max) {
            if (K > (size_t)k_max) return TBPM_E_UNSUPPORTED;
            c.resize(K);
            for (size_t k = 0; k < K; ++k) c[k] = 2.0 * x[k].real() / (double)n;
            return TBPM_OK;
        }
    }
}

// Re sigma(omega) = norm (e^{-beta omega} - 1) / omega
//                   * int_0^T e^{-eta t} sin(omega t) 2 Im C(t) dt   (Sec. 2.7, Eq. AC)
// by the trapezoid rule on t_n = n tau, for each row of corr.
int ac_conductivity(const double *corr, int n_rows, int n_steps, double tau, double beta,
                    double eta, const double *omegas, int n_omega, double norm, double *sigma)
{
    if (!corr || !omegas || !sigma || n_rows < 1 || n_steps < 1 || n_omega < 1 ||
        !(tau > 0.0) || !(beta > 0.0) || !(eta >= 0.0))
        return TBPM_E_INVALID_ARG;
    for (int k = 0; k < n_omega; ++k)
        if (!(omegas[k] > 0.0) || !std::isfinite(omegas[k])) return TBPM_E_INVALID_ARG;
    for (int row = 0; row < n_rows; ++row) {
        const double *cr = corr + (size_t)row * (n_steps + 1) * 2;
        for (int k = 0; k < n_omega; ++k) {
            const double w = omegas[k];
            double acc = 0.0;
            for (int n = 1; n <= n_steps; ++n) {
                const double t = tau * n;
                const double g = exp(-eta * t) * sin(w * t) * 2.0 * cr[2 * n + 1];
                acc += (n == n_steps ? 0.5 : 1.0) * g;
            }
            sigma[(size_t)row * n_omega + k] = norm * (exp(-beta * w) - 1.0) / w * tau * acc;
        }
    }
    return TBPM_OK;
}

// Window w_n of the DOS transform (Sec. 2.4 names Hann, Gaussian and
// exponential windows without parameters): Hann (1 + cos(pi n/N))/2,
// Gaussian exp(-(3n/N)^2 / 2) (sigma = N/3), exponential exp(-4n/N).  The
// last sample enters with the trapezoid end weight 1/2.
double window_weight(int window, int n, int n_steps)
{
    const double x = (double)n / (double)n_steps;
    double w;
    switch (window) {
    case TBPM_WINDOW_GAUSSIAN: w = exp(-4.5 * x * x); break;
    case TBPM_WINDOW_EXPONENTIAL: w = exp(-4.0 * x); break;
    default: w = 0.5 * (1.0 + cos(M_PI * x)); break;
    }
    return n == n_steps ? 0.5 * w : w;
}

int dos_adjoint(const double *dl_dd, int n_e, int n_steps, double tau, double e_min,
                double e_max, int window, double *gbar_out)
{
    typedef std::complex<double> cd;
    const double de = (e_max - e_min) / n_e;
    std::vector<cd> acc(n_steps + 1, cd(0.0, 0.0));
    double s0 = 0.0;
    for (int k = 0; k < n_e; ++k) s0 += dl_dd[k];
    for (int k = 0; k < n_e; ++k) {
        const double E = e_min + (k + 0.5) * de;
        const cd step(cos(E * tau), -sin(E * tau));
        cd ph(1.0, 0.0);
        for (int n = 1; n <= n_steps; ++n) {
            if (n % 64 == 0) ph = cd(cos(E * tau * n), -sin(E * tau * n));
            else ph *= step;
            acc[n] += dl_dd[k] * ph;
        }
    }
    gbar_out[0] = tau / (2.0 * M_PI) * s0;
    gbar_out[1] = 0.0;
    for (int n = 1; n <= n_steps; ++n) {
        const double w = window_weight(window, n, n_steps);
        gbar_out[2 * n] = tau / M_PI * w * acc[n].real();
        gbar_out[2 * n + 1] = tau / M_PI * w * acc[n].imag();
    }
    return TBPM_OK;
}

}  // namespace tbpm

// ---- C ABI: host functions --------------------------------------------------

extern "C" int tbpm_bessel_coefficients(double z, double tol, int max_terms, double *J_out,
                                        int *n_terms)
{
    return tbpm::bessel_miller(z, tol, max_terms, J_out, n_terms);
}

// DOS by Horner evaluation of the windowed sum at each energy:
//   S(E) = sum_{n=1}^{N} w_n C_n u^n,  u = exp(i E tau)  (w_N with the end weight 1/2),
//   D(E) = (tau / pi) (Re C_0 / 2 + Re S(E)).
extern "C" int tbpm_dos(const double *corr, int n_steps, double tau, int window,
                        double e_min, double e_max, int n_e, double *energies_out,
                        double *dos_out)
{
    if (!corr || n_steps < 1 || !(tau > 0.0) || !(e_max > e_min) || n_e < 1 ||
        !energies_out || !dos_out)
        return TBPM_E_INVALID_ARG;
    if (window != TBPM_WINDOW_HANN && window != TBPM_WINDOW_GAUSSIAN &&
        window != TBPM_WINDOW_EXPONENTIAL)
        return TBPM_E_UNSUPPORTED;
    typedef std::complex<double> cd;
    std::vector<cd> wc(n_steps + 1);
    for (int n = 1; n <= n_steps; ++n)
        wc[n] = tbpm::window_weight(window, n, n_steps) * cd(corr[2 * n], corr[2 * n + 1]);
    const double de = (e_max - e_min) / n_e;
    const double c0 = 0.5 * corr[0];
#pragma omp parallel for schedule(static)
    for (int k = 0; k < n_e; ++k) {
        double E = e_min + (k + 0.5) * de;
        cd u(cos(E * tau), sin(E * tau));
        cd s(0.0, 0.0);
        for (int n = n_steps; n >= 1; --n) s = (s + wc[n]) * u;
        energies_out[k] = E;
        dos_out[k] = tau / M_PI * (c0 + s.real());
    }
    return TBPM_OK;
}

extern "C" int tbpm_dos_adjoint(const double *dl_dd, int n_e, int n_steps, double tau,
                                int window, double e_min, double e_max, double *gbar_out)
{
    if (!dl_dd || n_e < 1 || n_steps < 1 || !(tau > 0.0) || !(e_max > e_min) || !gbar_out)
        return TBPM_E_INVALID_ARG;
    if (window != TBPM_WINDOW_HANN && window != TBPM_WINDOW_GAUSSIAN &&
        window != TBPM_WINDOW_EXPONENTIAL)
        return TBPM_E_UNSUPPORTED;
    return tbpm::dos_adjoint(dl_dd, n_e, n_steps, tau, e_min, e_max, window, gbar_out);
}

extern "C" int tbpm_fermi_coefficients(double beta_s, double mu_s, int k_max, double *c_out,
                                       int *n_terms)
{
    if (!n_terms || k_max < 1) return TBPM_E_INVALID_ARG;
    std::vector<double> c;
    const int rc = tbpm::fermi_coefficients(beta_s, mu_s, 1e-15, k_max, c);
    if (rc) return rc;
    *n_terms = (int)c.size();
    if (c_out) memcpy(c_out, c.data(), c.size() * sizeof(double));
    return TBPM_OK;
}

extern "C" int tbpm_ac_conductivity(const double *corr, int n_rows, int n_steps, double tau,
                                    double beta, double eta, const double *omegas, int n_omega,
                                    double norm, double *sigma_out)
{
    return tbpm::ac_conductivity(corr, n_rows, n_steps, tau, beta, eta, omegas, n_omega, norm,
                                 sigma_out);
}
