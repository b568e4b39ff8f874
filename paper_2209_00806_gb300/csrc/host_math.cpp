// Host FP64 pieces of the TBPM path: the Bessel coefficient table of the
// Chebyshev expansion (Sec. 2.2) and the windowed Fourier transform of the
// correlation into the DOS (Sec. 2.4, Eq. dos_tbpm).
#include <math.h>
#include <string.h>

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
int dos_adjoint(const double *dl_dd, int n_e, int n_steps, double tau, double e_min,
                double e_max, double *gbar_out)
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
        for (int n = 1; n < n_steps; ++n) {
            if (n % 64 == 0) ph = cd(cos(E * tau * n), -sin(E * tau * n));
            else ph *= step;
            acc[n] += dl_dd[k] * ph;
        }
    }
    gbar_out[0] = tau / (2.0 * M_PI) * s0;
    gbar_out[1] = 0.0;
    for (int n = 1; n < n_steps; ++n) {
        const double w = 0.5 * (1.0 + cos(M_PI * (double)n / (double)n_steps));
        gbar_out[2 * n] = tau / M_PI * w * acc[n].real();
        gbar_out[2 * n + 1] = tau / M_PI * w * acc[n].imag();
    }
    gbar_out[2 * n_steps] = 0.0;
    gbar_out[2 * n_steps + 1] = 0.0;
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
//   S(E) = sum_{n=1}^{N-1} w_n C_n u^n,  u = exp(i E tau),
//   D(E) = (tau / pi) (Re C_0 / 2 + Re S(E)).
extern "C" int tbpm_dos(const double *corr, int n_steps, double tau, int window,
                        double e_min, double e_max, int n_e, double *energies_out,
                        double *dos_out)
{
    if (!corr || n_steps < 1 || !(tau > 0.0) || !(e_max > e_min) || n_e < 1 ||
        !energies_out || !dos_out)
        return TBPM_E_INVALID_ARG;
    if (window != TBPM_WINDOW_HANN) return TBPM_E_UNSUPPORTED;
    typedef std::complex<double> cd;
    std::vector<cd> wc(n_steps);
    for (int n = 1; n < n_steps; ++n) {
        double w = 0.5 * (1.0 + cos(M_PI * (double)n / (double)n_steps));
        wc[n] = w * cd(corr[2 * n], corr[2 * n + 1]);
    }
    const double de = (e_max - e_min) / n_e;
    const double c0 = 0.5 * corr[0];
#pragma omp parallel for schedule(static)
    for (int k = 0; k < n_e; ++k) {
        double E = e_min + (k + 0.5) * de;
        cd u(cos(E * tau), sin(E * tau));
        cd s(0.0, 0.0);
        for (int n = n_steps - 1; n >= 1; --n) s = (s + wc[n]) * u;
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
    if (window != TBPM_WINDOW_HANN) return TBPM_E_UNSUPPORTED;
    return tbpm::dos_adjoint(dl_dd, n_e, n_steps, tau, e_min, e_max, gbar_out);
}
