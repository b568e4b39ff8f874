/*
 * Plain CPU FP64 oracle of the TBPM time-evolution path.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the library's product path may call,
 * link or load this file; only the tests, the package's smoke check and the
 * benchmark's CPU-baseline leg use it.  It shares no code with the CUDA
 * library: it is written straight from the paper's equations, slowly and
 * plainly, so that a reader can check it against the paper by eye.
 *
 *   Hamiltonian (Sec. 2.1, Eq. ham_mat_finite, and the hopping convention of
 *   Sec. 4.1): H_ii = eps_i, H_ij = t for a listed bond (i, j, t) and
 *   H_ji = conj(t) for its implied conjugate.  The matrix is never assembled:
 *   H x is evaluated as the defining sum over the bond list.
 *   Rescaling (Sec. 2.2): H~ = H / s.
 *   Propagation (Sec. 2.2, Eq. psi_t and the modified Chebyshev recurrence):
 *   psi(t + tau) = [J_0(z) T^_0 + 2 sum_{m>=1} J_m(z) T^_m] psi(t), z = s tau,
 *   T^_0 = 1, T^_1 = -i H~, T^_{m+1} = -2 i H~ T^_m + T^_{m-1}.
 *   Correlation (Sec. 2.2, Eq. corr_dos): C_n = <psi_0 | psi(n tau)>.
 *   DOS (Sec. 2.4, Eq. dos_tbpm) with a one-sided Hann window, evaluated by
 *   direct numerical integration (the paper allows either an FFT or a direct
 *   integral).
 *
 * Readings of points the paper leaves open (the same list is kept with the
 * design notes): the series is cut at the first m > z with |J_m(z)| < 1e-15;
 * C has n_steps + 1 samples C_0 .. C_{n_steps}; the DOS integral uses the
 * trapezoid rule on [0, n_steps tau] with C(-t) = conj C(t) and window
 * w_n = (1 + cos(pi n / n_steps)) / 2, at bin centres.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_OK 0
#define ORACLE_E_ARG -1
#define ORACLE_E_RANGE -2
#define ORACLE_E_NOMEM -3

/* Bessel function of the first kind J_m(z) by its ascending power series
 *   J_m(z) = sum_{k>=0} (-1)^k (z/2)^(2k+m) / (k! (k+m)!),
 * summed until the terms no longer change the sum.  The alternating terms
 * peak near k ~ z/2 at about exp(z)/(2 pi z); for z <= 4 the cancellation
 * costs less than one decimal digit, so the oracle refuses larger z. */
int oracle_bessel(double z, int m_max, double *J)
{
    if (!(z >= 0.0) || z > 4.0 || m_max < 0 || !J)
        return ORACLE_E_RANGE;
    double h = 0.5 * z;
    for (int m = 0; m <= m_max; ++m) {
        double term = 1.0;
        for (int q = 1; q <= m; ++q)
            term *= h / (double)q;                  /* (z/2)^m / m! */
        double sum = term;
        for (int k = 0; k < 200; ++k) {
            term *= -(h * h) / ((double)(k + 1) * (double)(k + 1 + m));
            double next = sum + term;
            if (next == sum && k > (int)z)
                break;
            sum = next;
        }
        J[m] = sum;
    }
    return ORACLE_OK;
}

/* Compensated (Neumaier) running sum: the inner products below add up
 * millions of terms of equal size, where a plain running sum drifts by
 * ~1e-10; this keeps the sum exact to about one rounding. */
typedef struct {
    double s, c;
} oracle_sum;

static void sum_add(oracle_sum *k, double x)
{
    double t = k->s + x;
    if (fabs(k->s) >= fabs(x))
        k->c += (k->s - t) + x;
    else
        k->c += (x - t) + k->s;
    k->s = t;
}

static double sum_value(const oracle_sum *k) { return k->s + k->c; }

/* Number of Chebyshev coefficients M: the series keeps m = 0 .. M-1, where
 * M is the first m > z with |J_m(z)| < 1e-15. */
int oracle_n_terms(double z)
{
    double J[129];
    if (oracle_bessel(z, 128, J) != ORACLE_OK)
        return ORACLE_E_RANGE;
    for (int m = 0; m <= 128; ++m)
        if ((double)m > z && fabs(J[m]) < 1e-15)
            return m;
    return ORACLE_E_RANGE;
}

/* y = H~ x with H~ = H / s, by the defining sums over the onsite list and the
 * bond list (each bond contributes H_ij and its conjugate H_ji). */
void oracle_apply_h(int64_t n, const double *onsite, int64_t n_hop, const int64_t *hop_i,
                    const int64_t *hop_j, const double *hop_re, const double *hop_im,
                    double s, const double complex *x, double complex *y)
{
    for (int64_t i = 0; i < n; ++i)
        y[i] = onsite ? onsite[i] * x[i] : 0.0;
    for (int64_t b = 0; b < n_hop; ++b) {
        int64_t i = hop_i[b], j = hop_j[b];
        double complex t = hop_re[b] + I * (hop_im ? hop_im[b] : 0.0);
        y[i] += t * x[j];
        y[j] += conj(t) * x[i];
    }
    for (int64_t i = 0; i < n; ++i)
        y[i] /= s;
}

/* Largest Gershgorin row bound of H (eV): max_i |eps_i| + sum_j |H_ij|. */
double oracle_gershgorin(int64_t n, const double *onsite, int64_t n_hop,
                         const int64_t *hop_i, const int64_t *hop_j,
                         const double *hop_re, const double *hop_im)
{
    double *r = calloc((size_t)n, sizeof(double));
    if (!r)
        return -1.0;
    for (int64_t b = 0; b < n_hop; ++b) {
        double a = cabs(hop_re[b] + I * (hop_im ? hop_im[b] : 0.0));
        r[hop_i[b]] += a;
        r[hop_j[b]] += a;
    }
    double g = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        double v = r[i] + (onsite ? fabs(onsite[i]) : 0.0);
        if (v > g)
            g = v;
    }
    free(r);
    return g;
}

/* Random-phase initial state psi_i = exp(i theta_i) / sqrt(N) (Sec. 2.2,
 * Eq. ini_state: random complex a_i with sum |a_i|^2 = 1). */
void oracle_phase_state(int64_t n, const double *theta, double complex *psi)
{
    double a = 1.0 / sqrt((double)n);
    for (int64_t i = 0; i < n; ++i)
        psi[i] = a * (cos(theta[i]) + I * sin(theta[i]));
}

/* Propagate n_states states for n_steps steps of tau = z / s and record
 *   corr[p][k]  = <psi0_p | psi_p(k tau)>,  k = 0 .. n_steps
 *   norms[p][k] = <psi_p(k tau) | psi_p(k tau)>   (optional)
 *   psi_out[p]  = psi_p(n_steps tau)              (optional)
 * Each step is the paper's expansion with the modified recurrence, in the
 * paper's order: T^_0 = phi, T^_1 = -i H~ phi, acc = J_0 T^_0 + 2 J_1 T^_1,
 * then T^_{m+1} = -2 i H~ T^_m + T^_{m-1}, acc += 2 J_{m+1} T^_{m+1}. */
int oracle_propagate(int64_t n, const double *onsite, int64_t n_hop, const int64_t *hop_i,
                     const int64_t *hop_j, const double *hop_re, const double *hop_im,
                     double s, double z, int n_steps, int n_states,
                     const double complex *psi0, double complex *corr,
                     double *norms, double complex *psi_out)
{
    if (n <= 0 || n_steps < 0 || n_states <= 0 || !(s > 0.0) || !psi0 || !corr)
        return ORACLE_E_ARG;
    int M = oracle_n_terms(z);
    if (M < 2)
        return ORACLE_E_RANGE;
    double J[129];
    oracle_bessel(z, M, J);

    double complex *phi = malloc((size_t)n * sizeof(double complex));
    double complex *t0 = malloc((size_t)n * sizeof(double complex));
    double complex *t1 = malloc((size_t)n * sizeof(double complex));
    double complex *t2 = malloc((size_t)n * sizeof(double complex));
    double complex *acc = malloc((size_t)n * sizeof(double complex));
    if (!phi || !t0 || !t1 || !t2 || !acc) {
        free(phi); free(t0); free(t1); free(t2); free(acc);
        return ORACLE_E_NOMEM;
    }
    for (int p = 0; p < n_states; ++p) {
        const double complex *a = psi0 + (size_t)p * n;
        memcpy(phi, a, (size_t)n * sizeof(double complex));
        for (int k = 0; k <= n_steps; ++k) {
            if (k > 0) {
                /* one time step phi <- sum_m c_m T^_m phi */
                memcpy(t0, phi, (size_t)n * sizeof(double complex));
                oracle_apply_h(n, onsite, n_hop, hop_i, hop_j, hop_re, hop_im, s, t0, t1);
                for (int64_t i = 0; i < n; ++i) {
                    t1[i] *= -I;
                    acc[i] = J[0] * t0[i] + 2.0 * J[1] * t1[i];
                }
                for (int m = 2; m < M; ++m) {
                    oracle_apply_h(n, onsite, n_hop, hop_i, hop_j, hop_re, hop_im, s, t1, t2);
                    for (int64_t i = 0; i < n; ++i) {
                        t2[i] = -2.0 * I * t2[i] + t0[i];
                        acc[i] += 2.0 * J[m] * t2[i];
                    }
                    double complex *tmp = t0;
                    t0 = t1;
                    t1 = t2;
                    t2 = tmp;
                }
                memcpy(phi, acc, (size_t)n * sizeof(double complex));
            }
            /* C_k = sum_i conj(psi0_i) phi_i and <phi|phi>, each summed with
             * compensation */
            oracle_sum cre = {0, 0}, cim = {0, 0}, nn = {0, 0};
            for (int64_t i = 0; i < n; ++i) {
                double complex v = conj(a[i]) * phi[i];
                sum_add(&cre, creal(v));
                sum_add(&cim, cimag(v));
                sum_add(&nn, creal(phi[i]) * creal(phi[i]) + cimag(phi[i]) * cimag(phi[i]));
            }
            corr[(size_t)p * (n_steps + 1) + k] = sum_value(&cre) + I * sum_value(&cim);
            if (norms)
                norms[(size_t)p * (n_steps + 1) + k] = sum_value(&nn);
        }
        if (psi_out)
            memcpy(psi_out + (size_t)p * n, phi, (size_t)n * sizeof(double complex));
    }
    free(phi); free(t0); free(t1); free(t2); free(acc);
    return ORACLE_OK;
}

/* DOS from the state-averaged correlation (Sec. 2.4, Eq. dos_tbpm):
 *   D(E) = (1/2 pi) int e^{iEt} C(t) dt
 *        = (tau/pi) [ Re C_0 / 2 + sum_{n=1}^{N-1} w_n Re(e^{i E n tau} C_n) ],
 * using C(-t) = conj C(t), the trapezoid rule on [0, N tau] and the
 * one-sided Hann window w_n = (1 + cos(pi n / N)) / 2 (w_N = 0).  Energies
 * are the bin centres E_k = e_min + (k + 1/2)(e_max - e_min)/n_e. */
int oracle_dos(const double complex *corr, int n_steps, double tau, double e_min,
               double e_max, int n_e, double *energies, double *dos)
{
    if (n_steps < 1 || n_e < 1 || !(tau > 0.0) || !(e_max > e_min))
        return ORACLE_E_ARG;
    double de = (e_max - e_min) / n_e;
    for (int k = 0; k < n_e; ++k) {
        double E = e_min + (k + 0.5) * de;
        double sum = 0.5 * creal(corr[0]);
        for (int n = 1; n < n_steps; ++n) {
            double w = 0.5 * (1.0 + cos(M_PI * n / n_steps));
            double ph = E * n * tau;
            sum += w * creal((cos(ph) + I * sin(ph)) * corr[n]);
        }
        energies[k] = E;
        dos[k] = tau / M_PI * sum;
    }
    return ORACLE_OK;
}

/* ---- adjoint (gradients of a real loss of the correlations) -------------
 *
 * The loss L depends on the correlations C_n^(p) of every state p.  The
 * caller supplies gbar[p][n] = dL/dRe C_n + i dL/dIm C_n, so that
 * dL = sum Re(conj(gbar) dC).  Since C_n = <psi0|phi_n>, the adjoint source
 * of phi_n is gbar_n psi0, and the adjoint of the whole trajectory obeys
 *   Lambda_N = gbar_N psi0,  Lambda_n = gbar_n psi0 + P^dagger Lambda_{n+1},
 * with P = sum_m c_m T^_m(H~) the one-step propagator of Sec. 2.2.  Within a
 * step the paper's forward recurrence is differentiated in reverse order:
 *   mu_{M-1} = c_{M-1} Lambda,  mu_{M-2} = c_{M-2} Lambda + 2i H~ mu_{M-1},
 *   mu_m = c_m Lambda + 2i H~ mu_{m+1} + mu_{m+2}          (1 <= m <= M-3),
 *   mu_0 = c_0 Lambda + i H~ mu_1 + mu_2                     (= P^dagger Lambda),
 * and each product T^_m = -2i H~ T^_{m-1} + ... (factor -i for m = 1)
 * contributes, for a real symmetric change dH~ of entries (i, j) and (j, i),
 *   dL += g_m Im(conj(mu_{m,i}) T^_{m-1,j} + conj(mu_{m,j}) T^_{m-1,i}) dH~_ij,
 * g_m = 2 (m >= 2) or 1 (m = 1); a diagonal change gives
 * g_m Im(conj(mu_{m,i}) T^_{m-1,i}).  With H~ = H / s: dL/dt_b and
 * dL/deps_i carry a factor 1/s.  Real hoppings only.  Every phi_n is kept,
 * so this is for small systems. */
int oracle_gradient(int64_t n, const double *onsite, int64_t n_hop, const int64_t *hop_i,
                    const int64_t *hop_j, const double *hop_re, double s, double z,
                    int n_steps, int n_states, const double complex *psi0,
                    const double complex *gbar, double *grad_hop, double *grad_onsite)
{
    if (n <= 0 || n_steps < 0 || n_states <= 0 || !(s > 0.0) || !psi0 || !gbar ||
        !grad_hop || !grad_onsite)
        return ORACLE_E_ARG;
    int M = oracle_n_terms(z);
    if (M < 2)
        return ORACLE_E_RANGE;
    double J[129], c[129];
    oracle_bessel(z, M, J);
    c[0] = J[0];
    for (int m = 1; m < M; ++m)
        c[m] = 2.0 * J[m];

    size_t vec = (size_t)n * sizeof(double complex);
    double complex *traj = malloc(vec * (size_t)(n_steps + 1));
    double complex *T = malloc(vec * (size_t)M);
    double complex *mu = malloc(vec * (size_t)(M + 2));
    double complex *lam = malloc(vec);
    double complex *tmp = malloc(vec);
    if (!traj || !T || !mu || !lam || !tmp) {
        free(traj); free(T); free(mu); free(lam); free(tmp);
        return ORACLE_E_NOMEM;
    }
    for (int64_t b = 0; b < n_hop; ++b)
        grad_hop[b] = 0.0;
    for (int64_t i = 0; i < n; ++i)
        grad_onsite[i] = 0.0;

    for (int p = 0; p < n_states; ++p) {
        const double complex *a = psi0 + (size_t)p * n;
        const double complex *g = gbar + (size_t)p * (n_steps + 1);
        /* forward trajectory phi_0 .. phi_N */
        memcpy(traj, a, vec);
        for (int k = 0; k < n_steps; ++k) {
            double complex *phi = traj + (size_t)k * n, *nxt = traj + (size_t)(k + 1) * n;
            double complex *T0 = T, *T1 = T + n;
            memcpy(T0, phi, vec);
            oracle_apply_h(n, onsite, n_hop, hop_i, hop_j, hop_re, NULL, s, T0, T1);
            for (int64_t i = 0; i < n; ++i) {
                T1[i] *= -I;
                nxt[i] = c[0] * T0[i] + c[1] * T1[i];
            }
            for (int m = 2; m < M; ++m) {
                double complex *Tm = T + (size_t)m * n;
                oracle_apply_h(n, onsite, n_hop, hop_i, hop_j, hop_re, NULL, s,
                               T + (size_t)(m - 1) * n, Tm);
                for (int64_t i = 0; i < n; ++i) {
                    Tm[i] = -2.0 * I * Tm[i] + T[(size_t)(m - 2) * n + i];
                    nxt[i] += c[m] * Tm[i];
                }
            }
        }
        /* backward */
        for (int64_t i = 0; i < n; ++i)
            lam[i] = g[n_steps] * a[i];
        for (int k = n_steps - 1; k >= 0; --k) {
            const double complex *phi = traj + (size_t)k * n;
            /* the step's polynomials T^_0 .. T^_{M-1} */
            memcpy(T, phi, vec);
            oracle_apply_h(n, onsite, n_hop, hop_i, hop_j, hop_re, NULL, s, T, T + n);
            for (int64_t i = 0; i < n; ++i)
                T[n + i] *= -I;
            for (int m = 2; m < M; ++m) {
                double complex *Tm = T + (size_t)m * n;
                oracle_apply_h(n, onsite, n_hop, hop_i, hop_j, hop_re, NULL, s,
                               T + (size_t)(m - 1) * n, Tm);
                for (int64_t i = 0; i < n; ++i)
                    Tm[i] = -2.0 * I * Tm[i] + T[(size_t)(m - 2) * n + i];
            }
            /* mu_{M+1} = mu_M = 0, then the reverse recurrence */
            memset(mu + (size_t)M * n, 0, 2 * vec);
            for (int m = M - 1; m >= 0; --m) {
                double complex *mm = mu + (size_t)m * n;
                if (m == M - 1) {
                    for (int64_t i = 0; i < n; ++i)
                        mm[i] = c[m] * lam[i];
                    continue;
                }
                oracle_apply_h(n, onsite, n_hop, hop_i, hop_j, hop_re, NULL, s,
                               mu + (size_t)(m + 1) * n, tmp);
                double complex f = (m == 0) ? I : 2.0 * I;
                for (int64_t i = 0; i < n; ++i)
                    mm[i] = c[m] * lam[i] + f * tmp[i] + mu[(size_t)(m + 2) * n + i];
            }
            /* gradient contributions of T^_m = (-i g_m H~) T^_{m-1} + ... */
            for (int m = 1; m < M; ++m) {
                double gm = (m == 1) ? 1.0 : 2.0;
                const double complex *um = mu + (size_t)m * n;
                const double complex *tv = T + (size_t)(m - 1) * n;
                for (int64_t b = 0; b < n_hop; ++b) {
                    int64_t i = hop_i[b], j = hop_j[b];
                    grad_hop[b] += gm * cimag(conj(um[i]) * tv[j] + conj(um[j]) * tv[i]) / s;
                }
                for (int64_t i = 0; i < n; ++i)
                    grad_onsite[i] += gm * cimag(conj(um[i]) * tv[i]) / s;
            }
            /* Lambda_k = gbar_k psi0 + P^dagger Lambda_{k+1} */
            for (int64_t i = 0; i < n; ++i)
                lam[i] = g[k] * a[i] + mu[i];
        }
    }
    free(traj); free(T); free(mu); free(lam); free(tmp);
    return ORACLE_OK;
}

/* Adjoint of oracle_dos: given dL/dD_k for each energy bin, return
 * gbar_n = dL/dRe C_n + i dL/dIm C_n of the averaged correlation.  From
 * D_k = (tau/pi)[Re C_0 / 2 + sum_{n=1}^{N-1} w_n Re(e^{i E_k n tau} C_n)]:
 *   gbar_0 = (tau / 2 pi) sum_k dL/dD_k,
 *   gbar_n = (tau / pi) w_n sum_k dL/dD_k e^{-i E_k n tau}   (1 <= n < N),
 *   gbar_N = 0. */
int oracle_dos_adjoint(const double *dl_dd, int n_steps, double tau, double e_min,
                       double e_max, int n_e, double complex *gbar)
{
    if (n_steps < 1 || n_e < 1 || !(tau > 0.0) || !(e_max > e_min))
        return ORACLE_E_ARG;
    double de = (e_max - e_min) / n_e;
    double s0 = 0.0;
    for (int k = 0; k < n_e; ++k)
        s0 += dl_dd[k];
    gbar[0] = tau / (2.0 * M_PI) * s0;
    for (int n = 1; n < n_steps; ++n) {
        double w = 0.5 * (1.0 + cos(M_PI * n / n_steps));
        double complex acc = 0.0;
        for (int k = 0; k < n_e; ++k) {
            double ph = (e_min + (k + 0.5) * de) * n * tau;
            acc += dl_dd[k] * (cos(ph) - I * sin(ph));
        }
        gbar[n] = tau / M_PI * w * acc;
    }
    gbar[n_steps] = 0.0;
    return ORACLE_OK;
}
