/*
 * FP64 CPU oracle for the lattice evolution of arXiv:2006.15122
 * ("The Art of Simulating the Early Universe -- Part I").
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the
 * benchmark's CPU-baseline leg may load this file's library.  It shares no
 * code, header, table or constant with the CUDA library and imports nothing
 * from it.  It is written to be read against the paper: every function
 * follows one passage, in the paper's order and notation, in plain FP64,
 * with unmerged half-kicks and no fusion.
 *
 * Conventions (paper section 3.1):
 *   site n = (n1,n2,n3), linear index (n3*N + n2)*N + n1, n1 fastest;
 *   periodic boundary conditions in the three directions;
 *   program variables of section 4.1: phi~ = phi/f_star, d eta~ = a^-alpha w_star dt,
 *   dx~ = w_star dx, V~ = V/(f_star^2 w_star^2).
 *
 * Scalar sector (section 4): N_s real fields with momenta
 *   pi_i = a^{3-alpha} phi_i'           (Hamiltonian form, section 4.2.3)
 *   phi_i' = a^{-(3-alpha)} pi_i
 *   pi_i'  = K_i = a^{1+alpha} L[phi_i] - a^{3+alpha} dV/dphi_i
 *   L[f](n) = sum_k (f(n+k) + f(n-k) - 2 f(n)) / dx^2   (= sum_k D_k^- D_k^+ f)
 *   b' = K_a = (1/3)(fstar/m_p)^2 a^{1+2 alpha} [(alpha-2)E_K + alpha E_G + (alpha+1) E_V]
 *   E_K = sum_i <pi_i^2>/(2 a^6), E_G = sum_{i,k} <(D_k^+ phi_i)^2>/(2 a^2), E_V = <V>
 * Potential (section 8.1, program units): V = (lam/p)|phi|^p + (q/2) phi^2 chi^2.
 *
 * U(1) sector (section 5, compact formulation 5.3): complex phi, momentum
 * pi = a^{3-alpha} phi', link angles theta_i = e dx A_i (V_i = exp(-i theta_i)),
 * electric momenta piA_i = a^{1-alpha} F_0i.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_MAXF 2

typedef struct {
    int64_t N;     /* sites per dimension */
    int32_t Ns;    /* number of real scalar fields (1 or 2) */
    int32_t pexp;  /* exponent p of the inflaton term (2, 4 or 6) */
    double dx;     /* lattice spacing, program units */
    double alpha;  /* alpha-time exponent */
    double fmp2;   /* (fstar/m_p)^2; 0 means a static background (a = 1, b = 0) */
    double lam;    /* coefficient of (1/p)|phi|^p */
    double q;      /* coupling of (q/2) phi^2 chi^2 (only with Ns = 2) */
} orc_scalar_model;

static inline int64_t wrap(int64_t i, int64_t N) { return (i % N + N) % N; }
static inline int64_t site(int64_t N, int64_t x, int64_t y, int64_t z) { return (z * N + y) * N + x; }

static double ipow(double x, int k) {
    double r = 1.0;
    for (int i = 0; i < k; ++i) r *= x;
    return r;
}

/* ---------------------------------------------------------------- scalars */

/* Potential terms of section 8.1: V_1 = (lam/p)|phi|^p, V_2 = (q/2) phi^2 chi^2. */
static void potential_terms(const orc_scalar_model* m, double phi, double chi, double* v1, double* v2) {
    *v1 = m->lam / m->pexp * ipow(fabs(phi), m->pexp);
    *v2 = (m->Ns > 1) ? 0.5 * m->q * phi * phi * chi * chi : 0.0;
}

/* dV/dphi = lam |phi|^{p-2} phi + q chi^2 phi,   dV/dchi = q phi^2 chi (section 8.1). */
static void potential_gradient(const orc_scalar_model* m, double phi, double chi, double* dphi, double* dchi) {
    *dphi = m->lam * ipow(fabs(phi), m->pexp - 2) * phi;
    *dchi = 0.0;
    if (m->Ns > 1) {
        *dphi += m->q * chi * chi * phi;
        *dchi = m->q * phi * phi * chi;
    }
}

/* Kernel of the scalar momenta, section 4.2.3 (Hamiltonian form):
 * K_i(n) = a^{1+alpha} L[phi_i](n) - a^{3+alpha} dV/dphi_i(n). */
void orc_scalar_kernel(const orc_scalar_model* m, const double* phi, double a, double* K) {
    const int64_t N = m->N, V = N * N * N;
    const double idx2 = 1.0 / (m->dx * m->dx);
    const double a1 = pow(a, 1.0 + m->alpha), a3 = pow(a, 3.0 + m->alpha);
#pragma omp parallel for schedule(static)
    for (int64_t z = 0; z < N; ++z)
        for (int64_t y = 0; y < N; ++y)
            for (int64_t x = 0; x < N; ++x) {
                const int64_t n = site(N, x, y, z);
                const double f0 = phi[n], f1 = (m->Ns > 1) ? phi[V + n] : 0.0;
                double d0, d1;
                potential_gradient(m, f0, f1, &d0, &d1);
                for (int i = 0; i < m->Ns; ++i) {
                    const double* f = phi + (int64_t)i * V;
                    const double lap = (f[site(N, wrap(x + 1, N), y, z)] + f[site(N, wrap(x - 1, N), y, z)] +
                                        f[site(N, x, wrap(y + 1, N), z)] + f[site(N, x, wrap(y - 1, N), z)] +
                                        f[site(N, x, y, wrap(z + 1, N))] + f[site(N, x, y, wrap(z - 1, N))] -
                                        6.0 * f[n]) * idx2;
                    K[(int64_t)i * V + n] = a1 * lap - a3 * (i == 0 ? d0 : d1);
                }
            }
}

/* Energies of section 4.4.1 (with pi = a^{3-alpha} phi', so E_K carries a^-6).
 * out[0..1] = E_K per field, out[2..3] = E_G per field, out[4] = <V_1>, out[5] = <V_2>. */
void orc_scalar_energies(const orc_scalar_model* m, const double* phi, const double* pi, double a, double* out) {
    const int64_t N = m->N, V = N * N * N;
    double sk[ORC_MAXF] = {0, 0}, sg[ORC_MAXF] = {0, 0}, sv1 = 0, sv2 = 0;
    for (int i = 0; i < m->Ns; ++i) {
        const double* f = phi + (int64_t)i * V;
        const double* p = pi + (int64_t)i * V;
        double k = 0, g = 0;
#pragma omp parallel for reduction(+ : k, g) schedule(static)
        for (int64_t z = 0; z < N; ++z)
            for (int64_t y = 0; y < N; ++y)
                for (int64_t x = 0; x < N; ++x) {
                    const int64_t n = site(N, x, y, z);
                    const double gx = (f[site(N, wrap(x + 1, N), y, z)] - f[n]) / m->dx;
                    const double gy = (f[site(N, x, wrap(y + 1, N), z)] - f[n]) / m->dx;
                    const double gz = (f[site(N, x, y, wrap(z + 1, N))] - f[n]) / m->dx;
                    k += p[n] * p[n];
                    g += gx * gx + gy * gy + gz * gz;
                }
        sk[i] = k;
        sg[i] = g;
    }
#pragma omp parallel for reduction(+ : sv1, sv2) schedule(static)
    for (int64_t n = 0; n < V; ++n) {
        double v1, v2;
        potential_terms(m, phi[n], m->Ns > 1 ? phi[V + n] : 0.0, &v1, &v2);
        sv1 += v1;
        sv2 += v2;
    }
    const double a6 = pow(a, 6.0), a2 = a * a;
    for (int i = 0; i < ORC_MAXF; ++i) {
        out[i] = sk[i] / V / (2.0 * a6);
        out[2 + i] = sg[i] / V / (2.0 * a2);
    }
    out[4] = sv1 / V;
    out[5] = sv2 / V;
}

/* Scale-factor kernel K_a of section 4.3.2 from total E_K, E_G, E_V. */
static double Ka_scalar(const orc_scalar_model* m, double a, double EK, double EG, double EV) {
    return m->fmp2 / 3.0 * pow(a, 1.0 + 2.0 * m->alpha) *
           ((m->alpha - 2.0) * EK + m->alpha * EG + (m->alpha + 1.0) * EV);
}

static void totals(const double* E, double* EK, double* EG, double* EV) {
    *EK = E[0] + E[1];
    *EG = E[2] + E[3];
    *EV = E[4] + E[5];
}

double orc_scalar_Ka(const orc_scalar_model* m, double a, const double* E) {
    double EK, EG, EV;
    totals(E, &EK, &EG, &EV);
    return Ka_scalar(m, a, EK, EG, EV);
}

/* Right-hand side of the Hubble constraint b^2 = (1/3)(fstar/m_p)^2 a^{2(alpha+1)} (E_K+E_G+E_V). */
double orc_scalar_hubble_rhs(const orc_scalar_model* m, double a, const double* E) {
    double EK, EG, EV;
    totals(E, &EK, &EG, &EV);
    return m->fmp2 / 3.0 * pow(a, 2.0 * (m->alpha + 1.0)) * (EK + EG + EV);
}

static void kick(const orc_scalar_model* m, const double* phi, double* pi, double a, double h, double* K) {
    const int64_t V = m->N * m->N * m->N;
    orc_scalar_kernel(m, phi, a, K);
    for (int64_t n = 0; n < (int64_t)m->Ns * V; ++n) pi[n] += h * K[n];
}

static void drift(const orc_scalar_model* m, double* phi, const double* pi, double c) {
    const int64_t V = m->N * m->N * m->N;
    for (int64_t n = 0; n < (int64_t)m->Ns * V; ++n) phi[n] += c * pi[n];
}

/* One full step of the Yoshida-composed velocity-Verlet integrator VVn for
 * scalars in a self-consistently expanding background (section 4.3.2).  For
 * each sub-step p = 1..s with weight w_p:
 *   b_1/2   = b + w_p dt/2 K_a[a, E(p-1)]
 *   pi_1/2  = pi + w_p dt/2 K[a, phi]
 *   a_1/2   = a + b_1/2 w_p dt/2
 *   phi     = phi + w_p dt pi_1/2 a_1/2^{-(3-alpha)}
 *   a       = a_1/2 + b_1/2 w_p dt/2
 *   pi      = pi_1/2 + w_p dt/2 K[a, phi]
 *   b       = b_1/2 + w_p dt/2 K_a[a, E(p)]
 * s = 1, w = {1} is VV2 (section 4.2.3).  E(p-1) is the energy of the state
 * before the sub-step, E(p) the one after it. */
void orc_scalar_vv_step(const orc_scalar_model* m, int s, const double* w, double dt,
                        double* phi, double* pi, double* a, double* b) {
    const int64_t V = m->N * m->N * m->N;
    double* K = (double*)malloc(sizeof(double) * (size_t)(m->Ns * V));
    double E[6];
    orc_scalar_energies(m, phi, pi, *a, E);
    for (int p = 0; p < s; ++p) {
        const double h = w[p] * dt;
        const double bh = *b + 0.5 * h * orc_scalar_Ka(m, *a, E);
        kick(m, phi, pi, *a, 0.5 * h, K);
        const double ah = *a + 0.5 * h * bh;
        drift(m, phi, pi, h * pow(ah, -(3.0 - m->alpha)));
        *a = ah + 0.5 * h * bh;
        kick(m, phi, pi, *a, 0.5 * h, K);
        orc_scalar_energies(m, phi, pi, *a, E);
        *b = bh + 0.5 * h * orc_scalar_Ka(m, *a, E);
    }
    free(K);
}

/* Scheme III of section 4.2.1 needs E_K at n+1/2, which contains a_{n+1/2} =
 * a_n + dt b_{n+1/2}/2, while b_{n+1/2} itself depends on that E_K through the
 * averaged kinetic energy.  The paper leaves this scalar fixed point implicit;
 * it is solved here by plain fixed-point iteration to round-off, with
 * S = sum_i <pi_i^2> at n+1/2 fixed. */
static double lf3_solve_b(const orc_scalar_model* m, double dt, double a, double bm, double EKm, double S,
                          double EG, double EV, double* EKp_out) {
    double bp = bm, EKp = 0.0;
    for (int it = 0; it < 200; ++it) {
        const double ah = a + 0.5 * dt * bp;
        EKp = S / (2.0 * pow(ah, 6.0));
        const double EKbar = 0.5 * (EKm + EKp);
        const double bn = bm + dt * Ka_scalar(m, a, EKbar, EG, EV);
        const double d = fabs(bn - bp);
        bp = bn;
        if (d <= 1e-17 * fabs(bn) || d == 0.0) break;
    }
    const double ah = a + 0.5 * dt * bp;
    *EKp_out = S / (2.0 * pow(ah, 6.0));
    return bp;
}

/* Start scheme III from a synchronized state (phi, pi, a, b at eta_0): the
 * half-step-behind momenta are taken with a backward half kick,
 * pi_{-1/2} = pi - dt/2 K[a, phi] and b_{-1/2} = b - dt/2 K_a[a, E].
 * Returns E_K at -1/2 in *EKm, with a_{-1/2} = a - dt b_{-1/2}/2. */
void orc_scalar_lf3_prepare(const orc_scalar_model* m, double dt, const double* phi, double* pi, double a,
                            double* b, double* EKm) {
    const int64_t V = m->N * m->N * m->N;
    double* K = (double*)malloc(sizeof(double) * (size_t)(m->Ns * V));
    double E[6];
    orc_scalar_energies(m, phi, pi, a, E);
    *b = *b - 0.5 * dt * orc_scalar_Ka(m, a, E);
    kick(m, phi, pi, a, -0.5 * dt, K);
    const double ahm = a - 0.5 * dt * (*b);
    double S = 0.0;
    for (int64_t n = 0; n < (int64_t)m->Ns * V; ++n) S += pi[n] * pi[n];
    *EKm = S / V / (2.0 * pow(ahm, 6.0));
    free(K);
}

/* One step of staggered leapfrog scheme III (section 4.2.1), state
 * (phi_n, a_n) at integer and (pi_{n-1/2}, b_{n-1/2}) at half-integer time:
 *   pi_{+1/2} = pi_{-1/2} + dt K[a, phi]
 *   b_{+1/2}  = b_{-1/2} + dt (1/3)(fstar/m_p)^2 a^{1+2alpha}[(alpha-2) <E_K> + alpha E_G + (alpha+1) E_V]
 *   a_{+1}    = a + dt b_{+1/2},  a_{+1/2} = (a + a_{+1})/2
 *   phi_{+1}  = phi + dt pi_{+1/2} a_{+1/2}^{-(3-alpha)}
 * with <E_K> the average of E_K at -1/2 and +1/2.  *EKm carries E_K at the
 * previous half step in and the new one out.  diag (may be NULL) receives
 * {E_G(n), E_V(n), E_K(n+1/2), a_{n+1/2}, b_{n+1/2}}. */
void orc_scalar_lf3_step(const orc_scalar_model* m, double dt, double* phi, double* pi, double* a, double* b,
                         double* EKm, double* diag) {
    const int64_t V = m->N * m->N * m->N;
    double* K = (double*)malloc(sizeof(double) * (size_t)(m->Ns * V));
    double E[6];
    orc_scalar_energies(m, phi, pi, *a, E); /* E_G, E_V at n (E_K entries unused) */
    const double EG = E[2] + E[3], EV = E[4] + E[5];
    kick(m, phi, pi, *a, dt, K);
    double S = 0.0;
    for (int64_t n = 0; n < (int64_t)m->Ns * V; ++n) S += pi[n] * pi[n];
    S /= (double)V;
    double EKp;
    const double bp = lf3_solve_b(m, dt, *a, *b, *EKm, S, EG, EV, &EKp);
    const double an = *a + dt * bp;
    const double ah = 0.5 * (*a + an);
    drift(m, phi, pi, dt * pow(ah, -(3.0 - m->alpha)));
    if (diag) {
        diag[0] = EG;
        diag[1] = EV;
        diag[2] = EKp;
        diag[3] = ah;
        diag[4] = bp;
    }
    *a = an;
    *b = bp;
    *EKm = EKp;
    free(K);
}

/* ------------------------------------------------------------------- U(1) */

typedef struct {
    int64_t N;
    double dx, alpha, fmp2;
    double lam, v2; /* V = (lam/4)(|phi|^2 - v2)^2, or the monomial inflaton below */
    double e;       /* gauge coupling g_A Q_A */
    double kappa;   /* (omega_star/f_star)^2 */
    int32_t pot;    /* 0: Abelian-Higgs; 1: V = (lam/p)(2|phi|^2)^(p/2) (section 8.1 with |phi| -> sqrt(2)|phi|) */
    int32_t p;
    int32_t noncompact; /* 1: the non-compact gauge kinetics of section 5.2 */
    int32_t pad;
} orc_u1_model;

/* Magnetic part of the gauge field's action per plaquette angle theta_ij and
 * its derivative: compact (section 5.3) 1 - cos theta_ij and sin theta_ij;
 * non-compact (section 5.2) (D_i^+ A_j - D_j^+ A_i)^2 (e dx^2)^2 / 2 = theta_ij^2 / 2
 * and theta_ij (the angles theta_i = e dx A_i are then plain real fields). */
static double u1_mag_energy(const orc_u1_model* m, double t) { return m->noncompact ? 0.5 * t * t : 1.0 - cos(t); }
static double u1_mag_force(const orc_u1_model* m, double t) { return m->noncompact ? t : sin(t); }

/* V(|phi|^2) of the charged scalar and V' = dV/d|phi|^2 (so that dV/dphi* = V' phi). */
static double gauge_potential(int pot, int p, double lam, double v2, double mod2, double* dv) {
    if (pot == 0) {
        *dv = 0.5 * lam * (mod2 - v2);
        return 0.25 * lam * (mod2 - v2) * (mod2 - v2);
    }
    const double s = 2.0 * mod2;
    *dv = lam * pow(s, 0.5 * p - 1.0);
    return lam / p * pow(s, 0.5 * p);
}

/* Plaquette angle theta_ij(n) = theta_i(n) + theta_j(n+i) - theta_i(n+j) - theta_j(n),
 * so that V_ij = V_i V_{j,+i} V*_{i,+j} V*_j = exp(-i theta_ij) (U(1) toolkit, section 3.2.2). */
static double plaq(const orc_u1_model* m, const double* th, int i, int j, int64_t x, int64_t y, int64_t z) {
    const int64_t N = m->N, V = N * N * N;
    int64_t c[3] = {x, y, z};
    int64_t ci[3] = {x, y, z}, cj[3] = {x, y, z};
    ci[i] = wrap(ci[i] + 1, N);
    cj[j] = wrap(cj[j] + 1, N);
    const double* ti = th + (int64_t)i * V;
    const double* tj = th + (int64_t)j * V;
    return ti[site(N, c[0], c[1], c[2])] + tj[site(N, ci[0], ci[1], ci[2])] - ti[site(N, cj[0], cj[1], cj[2])] -
           tj[site(N, c[0], c[1], c[2])];
}

/* Kernels of the compact U(1) formulation (section 5.3):
 * K_phi  = -a^{3+alpha} dV/dphi* + a^{1+alpha} sum_i D_i^- D_i^+ phi,
 *          D_i^- D_i^+ phi = (V_i phi(n+i) - 2 phi + V_i*(n-i) phi(n-i))/dx^2,
 *          dV/dphi* = (lam/2)(|phi|^2 - v2) phi;
 * K_A,i = a^{1+alpha} (2e/dx)(1/kappa) Im[phi*(n) V_i(n) phi(n+i)]
 *        + a^{alpha-1}/(e dx^3) sum_{j!=i} [Im V_ij(n) - Im V_ij(n-j)].
 * phi is stored as (re, im) planes; K_phi likewise. */
void orc_u1_kernels(const orc_u1_model* m, const double* phi, const double* th, double a, double* Kphi,
                    double* KA) {
    const int64_t N = m->N, V = N * N * N;
    const double a1 = pow(a, 1.0 + m->alpha), a3 = pow(a, 3.0 + m->alpha), am = pow(a, m->alpha - 1.0);
    const double dx = m->dx;
    const double* pr = phi;
    const double* pim = phi + V;
#pragma omp parallel for schedule(static)
    for (int64_t z = 0; z < N; ++z)
        for (int64_t y = 0; y < N; ++y)
            for (int64_t x = 0; x < N; ++x) {
                const int64_t n = site(N, x, y, z);
                const int64_t c[3] = {x, y, z};
                double lr = -6.0 * pr[n], li = -6.0 * pim[n];
                for (int i = 0; i < 3; ++i) {
                    int64_t cp[3] = {x, y, z}, cm[3] = {x, y, z};
                    cp[i] = wrap(c[i] + 1, N);
                    cm[i] = wrap(c[i] - 1, N);
                    const int64_t np = site(N, cp[0], cp[1], cp[2]), nm = site(N, cm[0], cm[1], cm[2]);
                    const double t = th[(int64_t)i * V + n], tm = th[(int64_t)i * V + nm];
                    /* V_i phi(n+i), V_i = cos t - i sin t */
                    const double ur = cos(t) * pr[np] + sin(t) * pim[np];
                    const double ui = cos(t) * pim[np] - sin(t) * pr[np];
                    /* V_i*(n-i) phi(n-i) */
                    const double wr = cos(tm) * pr[nm] - sin(tm) * pim[nm];
                    const double wi = cos(tm) * pim[nm] + sin(tm) * pr[nm];
                    lr += ur + wr;
                    li += ui + wi;
                    /* current: Im[phi*(n) V_i phi(n+i)] = pr*ui - pim*ur */
                    const double cur = pr[n] * ui - pim[n] * ur;
                    double mag = 0.0;
                    for (int j = 0; j < 3; ++j) {
                        if (j == i) continue;
                        int64_t cmj[3] = {x, y, z};
                        cmj[j] = wrap(c[j] - 1, N);
                        /* Im V_ij = -sin(theta_ij); non-compact: -theta_ij */
                        mag += -u1_mag_force(m, plaq(m, th, i, j, x, y, z)) +
                               u1_mag_force(m, plaq(m, th, i, j, cmj[0], cmj[1], cmj[2]));
                    }
                    KA[(int64_t)i * V + n] =
                        a1 * (2.0 * m->e / dx) / m->kappa * cur + am / (m->e * dx * dx * dx) * mag;
                }
                const double mod2 = pr[n] * pr[n] + pim[n] * pim[n];
                double dv;
                gauge_potential(m->pot, m->p, m->lam, m->v2, mod2, &dv);
                Kphi[n] = -a3 * dv * pr[n] + a1 * lr / (dx * dx);
                Kphi[V + n] = -a3 * dv * pim[n] + a1 * li / (dx * dx);
            }
}

/* Energies of section 5.4.1 (compact):
 * out[0] E_K^phi = <|pi|^2>/a^6,  out[1] E_G^phi = sum_i <|D_i^+ phi|^2>/a^2,
 * out[2] E_V = <V>,  out[3] E_K^A = kappa/(2a^4) sum_i <piA_i^2>,
 * out[4] E_G^A = kappa/(a^4 e^2 dx^4) sum_{i<j} <1 - cos theta_ij> (compact) or
 *        <theta_ij^2/2> (non-compact, section 5.2). */
void orc_u1_energies(const orc_u1_model* m, const double* phi, const double* pi, const double* th,
                     const double* piA, double a, double* out) {
    const int64_t N = m->N, V = N * N * N;
    const double* pr = phi;
    const double* pim = phi + V;
    double sk = 0, sg = 0, sv = 0, ska = 0, sga = 0;
#pragma omp parallel for reduction(+ : sk, sg, sv, ska, sga) schedule(static)
    for (int64_t z = 0; z < N; ++z)
        for (int64_t y = 0; y < N; ++y)
            for (int64_t x = 0; x < N; ++x) {
                const int64_t n = site(N, x, y, z);
                const int64_t c[3] = {x, y, z};
                sk += pi[n] * pi[n] + pi[V + n] * pi[V + n];
                const double mod2 = pr[n] * pr[n] + pim[n] * pim[n];
                double dv;
                sv += gauge_potential(m->pot, m->p, m->lam, m->v2, mod2, &dv);
                for (int i = 0; i < 3; ++i) {
                    int64_t cp[3] = {x, y, z};
                    cp[i] = wrap(c[i] + 1, N);
                    const int64_t np = site(N, cp[0], cp[1], cp[2]);
                    const double t = th[(int64_t)i * V + n];
                    const double ur = cos(t) * pr[np] + sin(t) * pim[np];
                    const double ui = cos(t) * pim[np] - sin(t) * pr[np];
                    const double dr = (ur - pr[n]) / m->dx, di = (ui - pim[n]) / m->dx;
                    sg += dr * dr + di * di;
                    ska += piA[(int64_t)i * V + n] * piA[(int64_t)i * V + n];
                    for (int j = i + 1; j < 3; ++j) sga += u1_mag_energy(m, plaq(m, th, i, j, x, y, z));
                }
            }
    const double a2 = a * a, a4 = a2 * a2, a6 = a4 * a2, dx4 = pow(m->dx, 4.0);
    out[0] = sk / V / a6;
    out[1] = sg / V / a2;
    out[2] = sv / V;
    out[3] = m->kappa * ska / V / (2.0 * a4);
    out[4] = m->kappa * sga / V / (a4 * m->e * m->e * dx4);
}

/* K_a with the U(1) weights of section 5.1: the gauge energies enter with (alpha-1). */
static double Ka_u1(const orc_u1_model* m, double a, double EKp, double EGp, double EV, double EKA, double EGA) {
    return m->fmp2 / 3.0 * pow(a, 2.0 * m->alpha + 1.0) *
           ((m->alpha - 2.0) * EKp + m->alpha * EGp + (m->alpha + 1.0) * EV + (m->alpha - 1.0) * (EKA + EGA));
}

double orc_u1_Ka(const orc_u1_model* m, double a, const double* E) {
    return Ka_u1(m, a, E[0], E[1], E[2], E[3], E[4]);
}

/* Gauss-law residual of the compact U(1) sector (section 5.2, discrete Gauss law):
 * G(n) = sum_i D_i^- piA_i(n) - (2e/kappa) Im[phi*(n) pi(n)].
 * The sign of the charge term follows from the kernels above (both follow
 * from one lattice action).  lhs/rhs receive the two terms per site; out[0] =
 * <G^2>, out[1] = <lhs^2>, out[2] = <rhs^2>. */
void orc_u1_gauss(const orc_u1_model* m, const double* phi, const double* pi, const double* piA, double* lhs,
                  double* rhs, double* out) {
    const int64_t N = m->N, V = N * N * N;
    double g2 = 0, l2 = 0, r2 = 0;
#pragma omp parallel for reduction(+ : g2, l2, r2) schedule(static)
    for (int64_t z = 0; z < N; ++z)
        for (int64_t y = 0; y < N; ++y)
            for (int64_t x = 0; x < N; ++x) {
                const int64_t n = site(N, x, y, z);
                const int64_t c[3] = {x, y, z};
                double div = 0.0;
                for (int i = 0; i < 3; ++i) {
                    int64_t cm[3] = {x, y, z};
                    cm[i] = wrap(c[i] - 1, N);
                    const int64_t nm = site(N, cm[0], cm[1], cm[2]);
                    div += (piA[(int64_t)i * V + n] - piA[(int64_t)i * V + nm]) / m->dx;
                }
                /* Im[phi* pi] = re(phi) im(pi) - im(phi) re(pi) */
                const double rho = phi[n] * pi[V + n] - phi[V + n] * pi[n];
                const double r = 2.0 * m->e / m->kappa * rho;
                if (lhs) lhs[n] = div;
                if (rhs) rhs[n] = r;
                g2 += (div - r) * (div - r);
                l2 += div * div;
                r2 += r * r;
            }
    out[0] = g2 / V;
    out[1] = l2 / V;
    out[2] = r2 / V;
}

/* Backward half kick that starts the compact staggered leapfrog from a
 * synchronized state: pi_{-1/2} = pi - dt/2 K_phi, piA_{-1/2} = piA - dt/2 K_A,
 * b_{-1/2} = b - dt/2 K_a[a, E].  *EKm receives E_K^phi + E_K^A at -1/2 with
 * a_{-1/2} = a - dt b_{-1/2}/2 (the two kinetic terms scale as a^-6 and a^-4). */
void orc_u1_lf_prepare(const orc_u1_model* m, double dt, const double* phi, double* pi, const double* th,
                       double* piA, double a, double* b, double* EKm_phi, double* EKm_A) {
    const int64_t V = m->N * m->N * m->N;
    double* Kp = (double*)malloc(sizeof(double) * (size_t)(2 * V));
    double* KA = (double*)malloc(sizeof(double) * (size_t)(3 * V));
    double E[5];
    orc_u1_energies(m, phi, pi, th, piA, a, E);
    *b -= 0.5 * dt * orc_u1_Ka(m, a, E);
    orc_u1_kernels(m, phi, th, a, Kp, KA);
    double sp = 0, sa = 0;
    for (int64_t n = 0; n < 2 * V; ++n) {
        pi[n] -= 0.5 * dt * Kp[n];
        sp += pi[n] * pi[n];
    }
    for (int64_t n = 0; n < 3 * V; ++n) {
        piA[n] -= 0.5 * dt * KA[n];
        sa += piA[n] * piA[n];
    }
    const double ahm = a - 0.5 * dt * (*b);
    *EKm_phi = sp / V / pow(ahm, 6.0);
    *EKm_A = m->kappa * sa / V / (2.0 * pow(ahm, 4.0));
    free(Kp);
    free(KA);
}

/* One step of the compact staggered leapfrog (section 5.3.1):
 *   pi_{+1/2}  = pi_{-1/2} + dt K_phi[a, phi, V]
 *   piA_{+1/2} = piA_{-1/2} + dt K_A[a, phi, V]
 *   b_{+1/2}   = b_{-1/2} + dt K_a[a, <E_K^phi>, E_G^phi, E_V, <E_K^A>, E_G^A]
 *   a_{+1}     = a + dt b_{+1/2}
 *   phi_{+1}   = phi + dt pi_{+1/2} / a_{+1/2}^{3-alpha}
 *   V_i,+1     = exp(-i e dx dt piA_{+1/2} / a_{+1/2}^{1-alpha}) V_i
 * The link drift is the exact exponential (theta_i += e dx dt piA/a^{1-alpha}),
 * which keeps |V_i| = 1; <E_K> averages the kinetic energies at -1/2 and +1/2
 * and the implicit dependence on a_{+1/2} is iterated to round-off. */
void orc_u1_lf_step(const orc_u1_model* m, double dt, double* phi, double* pi, double* th, double* piA,
                    double* a, double* b, double* EKm_phi, double* EKm_A) {
    const int64_t V = m->N * m->N * m->N;
    double* Kp = (double*)malloc(sizeof(double) * (size_t)(2 * V));
    double* KA = (double*)malloc(sizeof(double) * (size_t)(3 * V));
    double E[5];
    orc_u1_energies(m, phi, pi, th, piA, *a, E); /* E_G^phi, E_V, E_G^A at n */
    orc_u1_kernels(m, phi, th, *a, Kp, KA);
    double sp = 0, sa = 0;
    for (int64_t n = 0; n < 2 * V; ++n) {
        pi[n] += dt * Kp[n];
        sp += pi[n] * pi[n];
    }
    for (int64_t n = 0; n < 3 * V; ++n) {
        piA[n] += dt * KA[n];
        sa += piA[n] * piA[n];
    }
    sp /= (double)V;
    sa /= (double)V;
    double bp = *b, EKp = 0, EKA = 0;
    for (int it = 0; it < 200; ++it) {
        const double ah = *a + 0.5 * dt * bp;
        EKp = sp / pow(ah, 6.0);
        EKA = m->kappa * sa / (2.0 * pow(ah, 4.0));
        const double bn = *b + dt * Ka_u1(m, *a, 0.5 * (*EKm_phi + EKp), E[1], E[2], 0.5 * (*EKm_A + EKA), E[4]);
        const double d = fabs(bn - bp);
        bp = bn;
        if (d <= 1e-17 * fabs(bn) || d == 0.0) break;
    }
    const double an = *a + dt * bp;
    const double ah = 0.5 * (*a + an);
    EKp = sp / pow(ah, 6.0);
    EKA = m->kappa * sa / (2.0 * pow(ah, 4.0));
    const double cphi = dt * pow(ah, -(3.0 - m->alpha));
    const double cth = m->e * m->dx * dt * pow(ah, -(1.0 - m->alpha));
    for (int64_t n = 0; n < 2 * V; ++n) phi[n] += cphi * pi[n];
    for (int64_t n = 0; n < 3 * V; ++n) th[n] += cth * piA[n];
    *a = an;
    *b = bp;
    *EKm_phi = EKp;
    *EKm_A = EKA;
    free(Kp);
    free(KA);
}

/* One full step of the compact velocity-Verlet integrator VVn of the U(1)
 * sector (sections 5.3.2 and 5.3.3, Yoshida composition of section 4.3.2).
 * For each sub-step p = 1..s with h = w_p dt:
 *   pi_1/2   = pi  + h/2 K_phi[a, phi, V]
 *   piA_1/2  = piA + h/2 K_A[a, phi, V]
 *   b_1/2    = b   + h/2 K_a[a, E(p-1)]
 *   a'       = a + h b_1/2,            a_1/2 = (a + a')/2
 *   phi      = phi + h pi_1/2 / a_1/2^{3-alpha}
 *   V_i      = exp(-i e dx h piA_1/2 / a_1/2^{1-alpha}) V_i   (theta_i += e dx h piA_1/2 / a_1/2^{1-alpha})
 *   pi       = pi_1/2  + h/2 K_phi[a', phi, V]
 *   piA      = piA_1/2 + h/2 K_A[a', phi, V]
 *   b        = b_1/2   + h/2 K_a[a', E(p)]
 * E(p-1) are the energies before the sub-step, E(p) after it (with the
 * synchronized momenta).  The printed scalar drift of the n-th order scheme
 * carries dt without w_p; the composition needs h = w_p dt there as in the
 * link drift.  The link drift is the exact exponential, as in the leapfrog. */
void orc_u1_vv_step(const orc_u1_model* m, int s, const double* w, double dt, double* phi, double* pi, double* th,
                    double* piA, double* a, double* b) {
    const int64_t V = m->N * m->N * m->N;
    double* Kp = (double*)malloc(sizeof(double) * (size_t)(2 * V));
    double* KA = (double*)malloc(sizeof(double) * (size_t)(3 * V));
    double E[5];
    orc_u1_energies(m, phi, pi, th, piA, *a, E);
    for (int p = 0; p < s; ++p) {
        const double h = w[p] * dt;
        orc_u1_kernels(m, phi, th, *a, Kp, KA);
        for (int64_t n = 0; n < 2 * V; ++n) pi[n] += 0.5 * h * Kp[n];
        for (int64_t n = 0; n < 3 * V; ++n) piA[n] += 0.5 * h * KA[n];
        const double bh = *b + 0.5 * h * orc_u1_Ka(m, *a, E);
        const double an = *a + h * bh, ah = 0.5 * (*a + an);
        const double cphi = h * pow(ah, -(3.0 - m->alpha));
        const double cth = m->e * m->dx * h * pow(ah, -(1.0 - m->alpha));
        for (int64_t n = 0; n < 2 * V; ++n) phi[n] += cphi * pi[n];
        for (int64_t n = 0; n < 3 * V; ++n) th[n] += cth * piA[n];
        *a = an;
        orc_u1_kernels(m, phi, th, *a, Kp, KA);
        for (int64_t n = 0; n < 2 * V; ++n) pi[n] += 0.5 * h * Kp[n];
        for (int64_t n = 0; n < 3 * V; ++n) piA[n] += 0.5 * h * KA[n];
        orc_u1_energies(m, phi, pi, th, piA, *a, E);
        *b = bh + 0.5 * h * orc_u1_Ka(m, *a, E);
    }
    free(Kp);
    free(KA);
}

/* ------------------------------------------------ prescribed background */

/* Expansion sourced by an external fluid of constant equation of state w
 * (section 4.1): a(eta) = a0 (1 + H0 (eta - eta0)/p)^p with
 * p = 2/(3(1 + w) - 2 alpha) and H0 the program Hubble rate a'/a at eta0 = 0. */
typedef struct {
    double a0, H0, p;
} orc_fluid;

static double fluid_a(const orc_fluid* f, double t) { return f->a0 * pow(1.0 + f->H0 * t / f->p, f->p); }

/* One step of the Yoshida-composed velocity-Verlet VVn for scalars when the
 * scale factor is prescribed (section 4.1 with the integrator of section
 * 4.3.2): for each sub-step p with h = w_p dt,
 *   pi_1/2 = pi + h/2 K[a(t), phi]
 *   a_1/2  = (a(t) + a(t + h))/2
 *   phi    = phi + h pi_1/2 a_1/2^{-(3-alpha)}
 *   pi     = pi_1/2 + h/2 K[a(t + h), phi],   t <- t + h,
 * i.e. the self-consistent scheme with the b, a updates replaced by a(t). */
void orc_scalar_vv_step_fluid(const orc_scalar_model* m, const orc_fluid* f, int s, const double* w, double dt,
                              double* phi, double* pi, double* t) {
    const int64_t V = m->N * m->N * m->N;
    double* K = (double*)malloc(sizeof(double) * (size_t)(m->Ns * V));
    for (int p = 0; p < s; ++p) {
        const double h = w[p] * dt;
        const double a = fluid_a(f, *t), an = fluid_a(f, *t + h);
        kick(m, phi, pi, a, 0.5 * h, K);
        drift(m, phi, pi, h * pow(0.5 * (a + an), -(3.0 - m->alpha)));
        kick(m, phi, pi, an, 0.5 * h, K);
        *t += h;
    }
    free(K);
}

/* ----------------------------------------------------- explicit RK4 */

/* Right-hand side of the scalar system in the form of the explicit
 * Runge-Kutta scheme (section 4.3.1): velocities v = phi' (not the Hamiltonian
 * momenta), k_i = a^{-2(1-alpha)} L[phi_i] - (3-alpha)(b/a) v_i - a^{2 alpha} dV/dphi_i
 * and k_a = K_a[a, E_K, E_G, E_V] with E_K = sum_i <v_i^2>/(2 a^{2 alpha}). */
static double rk4_rhs(const orc_scalar_model* m, const double* phi, const double* v, double a, double b,
                      double* k) {
    const int64_t N = m->N, V = N * N * N;
    const double c1 = pow(a, -2.0 * (1.0 - m->alpha)), c2 = (3.0 - m->alpha) * b / a, c3 = pow(a, 2.0 * m->alpha);
    const double idx2 = 1.0 / (m->dx * m->dx);
    double sk = 0.0, sg = 0.0, sv = 0.0;
#pragma omp parallel for reduction(+ : sk, sg, sv) schedule(static)
    for (int64_t z = 0; z < N; ++z)
        for (int64_t y = 0; y < N; ++y)
            for (int64_t x = 0; x < N; ++x) {
                const int64_t n = site(N, x, y, z);
                const int64_t nb[6] = {site(N, wrap(x + 1, N), y, z), site(N, wrap(x - 1, N), y, z),
                                       site(N, x, wrap(y + 1, N), z), site(N, x, wrap(y - 1, N), z),
                                       site(N, x, y, wrap(z + 1, N)), site(N, x, y, wrap(z - 1, N))};
                double dV[ORC_MAXF] = {0.0, 0.0}, v1 = 0.0, v2 = 0.0;
                potential_gradient(m, phi[n], m->Ns > 1 ? phi[V + n] : 0.0, &dV[0], &dV[1]);
                potential_terms(m, phi[n], m->Ns > 1 ? phi[V + n] : 0.0, &v1, &v2);
                sv += v1 + v2;
                for (int f = 0; f < m->Ns; ++f) {
                    const double* p = phi + (int64_t)f * V;
                    double lap = -6.0 * p[n];
                    for (int j = 0; j < 6; ++j) lap += p[nb[j]];
                    lap *= idx2;
                    k[(int64_t)f * V + n] = c1 * lap - c2 * v[(int64_t)f * V + n] - c3 * dV[f];
                    sk += v[(int64_t)f * V + n] * v[(int64_t)f * V + n];
                    for (int j = 0; j < 6; j += 2) {
                        const double g = p[nb[j]] - p[n];
                        sg += g * g * idx2;
                    }
                }
            }
    const double EK = sk / V / (2.0 * pow(a, 2.0 * m->alpha)), EG = sg / V / (2.0 * a * a), EV = sv / V;
    return m->fmp2 / 3.0 * pow(a, 1.0 + 2.0 * m->alpha) * ((m->alpha - 2.0) * EK + m->alpha * EG + (m->alpha + 1.0) * EV);
}

/* One step of the explicit RK4 of section 4.3.1 (Butcher weights
 * b_21 = b_32 = 1/2, b_43 = 1 and 1/6, 1/3, 1/3, 1/6):
 *   stage p = 1..4:  y^(p) = y(n0) + dt b_{p,p-1} d^(p-1)   (y^(1) = y(n0)),
 *                    d^(p) = (v^(p), k^(p), b^(p), k_a^(p)) = derivatives of (phi, v, a, b) at y^(p),
 *   y(n0 + 1) = y(n0) + dt/6 (d^(1) + 2 d^(2) + 2 d^(3) + d^(4)).
 * phi and v (= phi', not the Hamiltonian momentum) are updated in place. */
void orc_scalar_rk4_step(const orc_scalar_model* m, double dt, double* phi, double* v, double* a, double* b) {
    const int64_t V = m->N * m->N * m->N, M = (int64_t)m->Ns * V;
    double* ps = (double*)malloc(sizeof(double) * (size_t)M);
    double* vs = (double*)malloc(sizeof(double) * (size_t)M);
    double* k = (double*)malloc(sizeof(double) * (size_t)M);
    double* acc_phi = (double*)malloc(sizeof(double) * (size_t)M);
    double* acc_v = (double*)malloc(sizeof(double) * (size_t)M);
    const double c[4] = {0.0, 0.5, 0.5, 1.0}, w[4] = {1.0 / 6.0, 1.0 / 3.0, 1.0 / 3.0, 1.0 / 6.0};
    memcpy(ps, phi, sizeof(double) * (size_t)M);
    memcpy(vs, v, sizeof(double) * (size_t)M);
    memcpy(acc_phi, phi, sizeof(double) * (size_t)M);
    memcpy(acc_v, v, sizeof(double) * (size_t)M);
    double ap = *a, bp = *b, ka = 0.0, acc_a = *a, acc_b = *b;
    for (int p = 0; p < 4; ++p) {
        if (p > 0) {
            for (int64_t n = 0; n < M; ++n) {
                const double vprev = vs[n];
                ps[n] = phi[n] + c[p] * dt * vprev;
                vs[n] = v[n] + c[p] * dt * k[n];
            }
            const double an = *a + c[p] * dt * bp, bn = *b + c[p] * dt * ka;
            ap = an;
            bp = bn;
        }
        ka = rk4_rhs(m, ps, vs, ap, bp, k);
        for (int64_t n = 0; n < M; ++n) {
            acc_phi[n] += w[p] * dt * vs[n];
            acc_v[n] += w[p] * dt * k[n];
        }
        acc_a += w[p] * dt * bp;
        acc_b += w[p] * dt * ka;
    }
    memcpy(phi, acc_phi, sizeof(double) * (size_t)M);
    memcpy(v, acc_v, sizeof(double) * (size_t)M);
    *a = acc_a;
    *b = acc_b;
    free(ps);
    free(vs);
    free(k);
    free(acc_phi);
    free(acc_v);
}

/* ------------------------------------------------------------------- SU(2) */

/* SU(2) sector with a Higgs doublet (section 6, compact formulation 6.2):
 *   Phi = (Phi_1, Phi_2) complex, stored as phi[0..3] = (Re Phi_1, Im Phi_1, Re Phi_2, Im Phi_2);
 *   pi = a^{3-alpha} Phi' in the same layout;
 *   links U_i = exp(-i g dx B_i^a sigma^a/2) stored as unit quaternions
 *     U = q0 + i (q1 sigma_1 + q2 sigma_2 + q3 sigma_3)  (SU(2) toolkit, section 3.2.3),
 *     u[(i*4 + c)*V + n] = q_c of U_i(n);
 *   piB_i^a = a^{1-alpha} G_0i^a, piB[(i*3 + a)*V + n].
 * Energies (section 6.3.1), kappa = (w_star/f_star)^2, g = g_B Q_B:
 *   E_K^Phi = <pi^dag pi>/a^6, E_G^Phi = sum_i <|D_i^+ Phi|^2>/a^2,
 *   D_i^+ Phi = (U_i Phi(n+i) - Phi(n))/dx, E_V = <(lam/4)(|Phi|^2 - v2)^2>,
 *   E_K^B = kappa/(2 a^4) sum_{a,i} <(piB_i^a)^2>,
 *   E_G^B = 2 kappa/(a^4 dx^4 g^2) sum_{i<j} <2 - Tr U_ij>  (per plaquette; the
 *           printed "2 - sum" is read as the sum over the three plaquettes of 2 - Tr),
 *   U_ij(n) = U_i(n) U_j(n+i) U_i^dag(n+j) U_j^dag(n).
 * Kernels: both follow from the Hamiltonian
 *   H = a^{alpha-3} sum pi^dag pi + a^{alpha-1}/(2 kappa) sum (kappa piB)^2 + W,
 *   W = a^{3+alpha} N^3 (E_G^Phi + E_V + E_G^B),
 * with (B, kappa piB) canonical and B varied along U -> exp(-i g dx dB^a sigma^a/2) U:
 *   K_Phi = -a^{3+alpha}(lam/2)(|Phi|^2 - v2) Phi + a^{1+alpha} sum_i (U_i Phi(n+i) - 2 Phi + U_i^dag(n-i) Phi(n-i))/dx^2,
 *   K_B,i^a = a^{1+alpha} (g/(kappa dx)) Im[Phi^dag sigma^a U_i Phi(n+i)]
 *           + a^{alpha-1} (2/(g dx^3)) sum_{j != i} (P_a[U_ij(n)] - P_a[U_j^dag(n-j) U_ij(n-j) U_j(n-j)]),
 * P_a the sigma^a component q_a of a quaternion (the projection that the printed
 * matrix form of the kernel leaves implicit).  Gauge invariance of H gives the
 * discrete Gauss law (conserved exactly by kicks and exact drifts):
 *   (1/dx) sum_i [piB_i(n) - U_i^dag(n-i) piB_i(n-i) U_i(n-i)]^a = (g/kappa) Im[Phi^dag sigma^a pi],
 * the transported term being the adjoint action on piB_i = piB_i^a sigma^a. */
typedef struct {
    int64_t N;
    double dx, alpha, fmp2, lam, v2, g, kappa;
    int32_t pot;  /* 0: (lam/4)(|Phi|^2 - v2)^2; 1: (lam/p)(2|Phi|^2)^(p/2) */
    int32_t p;
} orc_su2_model;

static void qmul(const double* p, const double* q, double* r) {
    /* (p0 + i p.s)(q0 + i q.s) = (p0 q0 - p.q) + i (p0 q + q0 p - p x q).s */
    const double r0 = p[0] * q[0] - p[1] * q[1] - p[2] * q[2] - p[3] * q[3];
    const double r1 = p[0] * q[1] + q[0] * p[1] - (p[2] * q[3] - p[3] * q[2]);
    const double r2 = p[0] * q[2] + q[0] * p[2] - (p[3] * q[1] - p[1] * q[3]);
    const double r3 = p[0] * q[3] + q[0] * p[3] - (p[1] * q[2] - p[2] * q[1]);
    r[0] = r0; r[1] = r1; r[2] = r2; r[3] = r3;
}
static void qconj(const double* q, double* r) { r[0] = q[0]; r[1] = -q[1]; r[2] = -q[2]; r[3] = -q[3]; }

/* U Phi with U = [[q0 + i q3, q2 + i q1], [-q2 + i q1, q0 - i q3]] acting on (Phi_1, Phi_2). */
static void umul(const double* q, const double* f, double* o) {
    const double ar = q[0], ai = q[3], br = q[2], bi = q[1], cr = -q[2], ci = q[1], dr = q[0], di = -q[3];
    o[0] = ar * f[0] - ai * f[1] + br * f[2] - bi * f[3];
    o[1] = ar * f[1] + ai * f[0] + br * f[3] + bi * f[2];
    o[2] = cr * f[0] - ci * f[1] + dr * f[2] - di * f[3];
    o[3] = cr * f[1] + ci * f[0] + dr * f[3] + di * f[2];
}

/* Im[x^dag sigma^a y] for doublets x, y, a = 1, 2, 3. */
static void im_sigma(const double* x, const double* y, double* out) {
    /* sigma_1 y = (y2, y1); sigma_2 y = (-i y2, i y1); sigma_3 y = (y1, -y2) */
    /* x^dag z = conj(x1) z1 + conj(x2) z2; Im = x1r z1i - x1i z1r + x2r z2i - x2i z2r */
    double z[4];
    z[0] = y[2]; z[1] = y[3]; z[2] = y[0]; z[3] = y[1];
    out[0] = x[0] * z[1] - x[1] * z[0] + x[2] * z[3] - x[3] * z[2];
    z[0] = y[3]; z[1] = -y[2]; z[2] = -y[1]; z[3] = y[0];
    out[1] = x[0] * z[1] - x[1] * z[0] + x[2] * z[3] - x[3] * z[2];
    z[0] = y[0]; z[1] = y[1]; z[2] = -y[2]; z[3] = -y[3];
    out[2] = x[0] * z[1] - x[1] * z[0] + x[2] * z[3] - x[3] * z[2];
}

static void getq(const double* u, int64_t V, int i, int64_t n, double* q) {
    for (int c = 0; c < 4; ++c) q[c] = u[((int64_t)i * 4 + c) * V + n];
}
static void getf(const double* f, int64_t V, int64_t n, double* o) {
    for (int c = 0; c < 4; ++c) o[c] = f[(int64_t)c * V + n];
}
static int64_t shift(int64_t N, int64_t x, int64_t y, int64_t z, int d, int s) {
    int64_t c[3] = {x, y, z};
    c[d] = wrap(c[d] + s, N);
    return site(N, c[0], c[1], c[2]);
}

/* plaquette U_ij at site n (coordinates x, y, z) */
static void plaquette(const orc_su2_model* m, const double* u, int i, int j, int64_t x, int64_t y, int64_t z,
                      double* P) {
    const int64_t N = m->N, V = N * N * N, n = site(N, x, y, z);
    double Ui[4], Uj_i[4], Ui_j[4], Uj[4], t1[4], t2[4], c1[4], c2[4];
    getq(u, V, i, n, Ui);
    getq(u, V, j, shift(N, x, y, z, i, 1), Uj_i);
    getq(u, V, i, shift(N, x, y, z, j, 1), Ui_j);
    getq(u, V, j, n, Uj);
    qconj(Ui_j, c1);
    qconj(Uj, c2);
    qmul(Ui, Uj_i, t1);
    qmul(t1, c1, t2);
    qmul(t2, c2, P);
}

void orc_su2_kernels(const orc_su2_model* m, const double* phi, const double* u, double a, double* Kp, double* KB) {
    const int64_t N = m->N, V = N * N * N;
    const double A1 = pow(a, 1.0 + m->alpha), A3 = pow(a, 3.0 + m->alpha), Am = pow(a, m->alpha - 1.0);
    const double idx2 = 1.0 / (m->dx * m->dx);
    const double cJ = m->g / (m->kappa * m->dx), cM = 2.0 / (m->g * m->dx * m->dx * m->dx);
#pragma omp parallel for schedule(static)
    for (int64_t z = 0; z < N; ++z)
        for (int64_t y = 0; y < N; ++y)
            for (int64_t x = 0; x < N; ++x) {
                const int64_t n = site(N, x, y, z);
                double f[4], lap[4] = {0, 0, 0, 0};
                getf(phi, V, n, f);
                for (int c = 0; c < 4; ++c) lap[c] = -6.0 * f[c];
                for (int i = 0; i < 3; ++i) {
                    const int64_t np = shift(N, x, y, z, i, 1), nm = shift(N, x, y, z, i, -1);
                    double q[4], qm[4], qmc[4], fp[4], fm[4], t[4], t2[4];
                    getq(u, V, i, n, q);
                    getq(u, V, i, nm, qm);
                    qconj(qm, qmc);
                    getf(phi, V, np, fp);
                    getf(phi, V, nm, fm);
                    umul(q, fp, t);
                    umul(qmc, fm, t2);
                    for (int c = 0; c < 4; ++c) lap[c] += t[c] + t2[c];
                    /* current term of K_B,i */
                    double js[3];
                    im_sigma(f, t, js);
                    /* magnetic term: plaquettes containing U_i(n) */
                    double mag[3] = {0, 0, 0};
                    for (int j = 0; j < 3; ++j) {
                        if (j == i) continue;
                        double P1[4], P2[4], Uj[4], Ujc[4], s1[4], Q[4];
                        plaquette(m, u, i, j, x, y, z, P1);
                        int64_t cm[3] = {x, y, z};
                        cm[j] = wrap(cm[j] - 1, N);
                        plaquette(m, u, i, j, cm[0], cm[1], cm[2], P2);
                        getq(u, V, j, site(N, cm[0], cm[1], cm[2]), Uj);
                        qconj(Uj, Ujc);
                        qmul(Ujc, P2, s1);
                        qmul(s1, Uj, Q);
                        for (int c = 0; c < 3; ++c) mag[c] += P1[c + 1] - Q[c + 1];
                    }
                    for (int c = 0; c < 3; ++c) KB[((int64_t)i * 3 + c) * V + n] = A1 * cJ * js[c] + Am * cM * mag[c];
                }
                const double mod2 = f[0] * f[0] + f[1] * f[1] + f[2] * f[2] + f[3] * f[3];
                double dv;
                gauge_potential(m->pot, m->p, m->lam, m->v2, mod2, &dv);
                for (int c = 0; c < 4; ++c) Kp[(int64_t)c * V + n] = -A3 * dv * f[c] + A1 * lap[c] * idx2;
            }
}

void orc_su2_energies(const orc_su2_model* m, const double* phi, const double* pi, const double* u,
                      const double* piB, double a, double* out) {
    const int64_t N = m->N, V = N * N * N;
    double sk = 0, sg = 0, sv = 0, skb = 0, sgb = 0;
#pragma omp parallel for reduction(+ : sk, sg, sv, skb, sgb) schedule(static)
    for (int64_t z = 0; z < N; ++z)
        for (int64_t y = 0; y < N; ++y)
            for (int64_t x = 0; x < N; ++x) {
                const int64_t n = site(N, x, y, z);
                double f[4], p[4];
                getf(phi, V, n, f);
                getf(pi, V, n, p);
                for (int c = 0; c < 4; ++c) sk += p[c] * p[c];
                const double mod2 = f[0] * f[0] + f[1] * f[1] + f[2] * f[2] + f[3] * f[3];
                double dv;
                sv += gauge_potential(m->pot, m->p, m->lam, m->v2, mod2, &dv);
                for (int i = 0; i < 3; ++i) {
                    double q[4], fp[4], t[4];
                    getq(u, V, i, n, q);
                    getf(phi, V, shift(N, x, y, z, i, 1), fp);
                    umul(q, fp, t);
                    for (int c = 0; c < 4; ++c) sg += (t[c] - f[c]) * (t[c] - f[c]);
                    for (int c = 0; c < 3; ++c) skb += piB[((int64_t)i * 3 + c) * V + n] * piB[((int64_t)i * 3 + c) * V + n];
                    for (int j = i + 1; j < 3; ++j) {
                        double P[4];
                        plaquette(m, u, i, j, x, y, z, P);
                        sgb += 2.0 - 2.0 * P[0];
                    }
                }
            }
    const double a2 = a * a, a4 = a2 * a2, a6 = a4 * a2, dx4 = m->dx * m->dx * m->dx * m->dx;
    out[0] = sk / V / a6;
    out[1] = sg / V / (m->dx * m->dx) / a2;
    out[2] = sv / V;
    out[3] = m->kappa * skb / V / (2.0 * a4);
    out[4] = 2.0 * m->kappa * sgb / V / (a4 * dx4 * m->g * m->g);
}

static double Ka_su2(const orc_su2_model* m, double a, const double* E) {
    return m->fmp2 / 3.0 * pow(a, 2.0 * m->alpha + 1.0) *
           ((m->alpha - 2.0) * E[0] + m->alpha * E[1] + (m->alpha + 1.0) * E[2] + (m->alpha - 1.0) * (E[3] + E[4]));
}

double orc_su2_Ka(const orc_su2_model* m, double a, const double* E) { return Ka_su2(m, a, E); }

/* Gauss residual: out = {<|G|^2>, <|lhs|^2>, <|rhs|^2>} summed over the three colours. */
void orc_su2_gauss(const orc_su2_model* m, const double* phi, const double* pi, const double* u, const double* piB,
                   double* out) {
    const int64_t N = m->N, V = N * N * N;
    double g2 = 0, l2 = 0, r2 = 0;
#pragma omp parallel for reduction(+ : g2, l2, r2) schedule(static)
    for (int64_t z = 0; z < N; ++z)
        for (int64_t y = 0; y < N; ++y)
            for (int64_t x = 0; x < N; ++x) {
                const int64_t n = site(N, x, y, z);
                double div[3] = {0, 0, 0};
                for (int i = 0; i < 3; ++i) {
                    const int64_t nm = shift(N, x, y, z, i, -1);
                    double q[4], qc[4], e[4] = {0, 0, 0, 0}, t[4], tr[4];
                    getq(u, V, i, nm, q);
                    qconj(q, qc);
                    for (int c = 0; c < 3; ++c) e[c + 1] = piB[((int64_t)i * 3 + c) * V + nm];
                    qmul(qc, e, t);
                    qmul(t, q, tr);
                    for (int c = 0; c < 3; ++c) div[c] += (piB[((int64_t)i * 3 + c) * V + n] - tr[c + 1]) / m->dx;
                }
                double f[4], p[4], rho[3];
                getf(phi, V, n, f);
                getf(pi, V, n, p);
                im_sigma(f, p, rho);
                for (int c = 0; c < 3; ++c) {
                    const double r = m->g / m->kappa * rho[c];
                    g2 += (div[c] - r) * (div[c] - r);
                    l2 += div[c] * div[c];
                    r2 += r * r;
                }
            }
    out[0] = g2 / V;
    out[1] = l2 / V;
    out[2] = r2 / V;
}

/* Link drift U_i <- exp(-i c piB_i^a sigma^a/2) U_i (the exact exponential of the
 * momentum drift of section 6.2, unitary for any step): quaternion
 * (cos(|c piB|/2), -sin(|c piB|/2) piB/|piB|) multiplied from the left. */
static void su2_drift(const orc_su2_model* m, double* phi, const double* pi, double* u, const double* piB,
                      double cphi, double cU) {
    const int64_t V = m->N * m->N * m->N;
    for (int64_t n = 0; n < 4 * V; ++n) phi[n] += cphi * pi[n];
    for (int i = 0; i < 3; ++i)
        for (int64_t n = 0; n < V; ++n) {
            double e[3], q[4], r[4], ex[4];
            for (int c = 0; c < 3; ++c) e[c] = cU * piB[((int64_t)i * 3 + c) * V + n];
            const double th = sqrt(e[0] * e[0] + e[1] * e[1] + e[2] * e[2]);
            const double s = th > 0 ? sin(0.5 * th) / th : 0.5;
            ex[0] = cos(0.5 * th);
            for (int c = 0; c < 3; ++c) ex[c + 1] = -s * e[c];
            getq(u, V, i, n, q);
            qmul(ex, q, r);
            for (int c = 0; c < 4; ++c) u[((int64_t)i * 4 + c) * V + n] = r[c];
        }
}

/* One full step of the SU(2) velocity-Verlet VVn (sections 6.2.2-6.2.3, the
 * Yoshida composition of section 4.3.2): for each sub-step with h = w_p dt,
 * half kicks of pi, piB and b with the kernels at the sub-step's start, a' = a + h b_1/2,
 * drifts with a_1/2 = (a + a')/2 (phi += h pi/a_1/2^{3-alpha}; links by the exact
 * exponential with c = g dx h/a_1/2^{1-alpha}), half kicks at the end and the closing
 * half kick of b with the energies after the sub-step. */
void orc_su2_vv_step(const orc_su2_model* m, int s, const double* w, double dt, double* phi, double* pi, double* u,
                     double* piB, double* a, double* b) {
    const int64_t V = m->N * m->N * m->N;
    double* Kp = (double*)malloc(sizeof(double) * (size_t)(4 * V));
    double* KB = (double*)malloc(sizeof(double) * (size_t)(9 * V));
    double E[5];
    orc_su2_energies(m, phi, pi, u, piB, *a, E);
    for (int p = 0; p < s; ++p) {
        const double h = w[p] * dt;
        orc_su2_kernels(m, phi, u, *a, Kp, KB);
        for (int64_t n = 0; n < 4 * V; ++n) pi[n] += 0.5 * h * Kp[n];
        for (int64_t n = 0; n < 9 * V; ++n) piB[n] += 0.5 * h * KB[n];
        const double bh = *b + 0.5 * h * Ka_su2(m, *a, E);
        const double an = *a + h * bh, ah = 0.5 * (*a + an);
        su2_drift(m, phi, pi, u, piB, h * pow(ah, -(3.0 - m->alpha)), m->g * m->dx * h * pow(ah, -(1.0 - m->alpha)));
        *a = an;
        orc_su2_kernels(m, phi, u, *a, Kp, KB);
        for (int64_t n = 0; n < 4 * V; ++n) pi[n] += 0.5 * h * Kp[n];
        for (int64_t n = 0; n < 9 * V; ++n) piB[n] += 0.5 * h * KB[n];
        orc_su2_energies(m, phi, pi, u, piB, *a, E);
        *b = bh + 0.5 * h * Ka_su2(m, *a, E);
    }
    free(Kp);
    free(KB);
}

/* ------------------------------------------------ SU(2) x U(1) + singlet */

/* The doublet of the working example of section 8.3: Phi charged under SU(2)
 * (links U_i, coupling g = g_B Q_B) and U(1) (link angles theta_i, V_i =
 * exp(-i theta_i), coupling eA = g_A Q_A), plus a real singlet chi with
 * V_int = q |Phi|^2 chi^2.  The parallel transporter of Phi is W_i = V_i U_i
 * (the phase commutes with U_i), so the covariant hopping terms of section 6
 * carry the extra phase and the two gauge sectors see the same hop:
 *   K_Phi   = -a^{3+alpha}(V'(|Phi|^2) + q chi^2) Phi
 *             + a^{1+alpha} sum_i (W_i Phi(n+i) - 2 Phi + W_i^dag(n-i) Phi(n-i))/dx^2,
 *   K_B,i^a = a^{1+alpha}(g/(kappa dx)) Im[Phi^dag sigma^a W_i Phi(n+i)] + (SU(2) magnetic term),
 *   K_A,i   = a^{1+alpha}(2 eA/(kappa dx)) Im[Phi^dag W_i Phi(n+i)]
 *             + a^{alpha-1}/(eA dx^3) sum_{j!=i} [Im V_ij(n) - Im V_ij(n-j)],
 *   K_chi   = -a^{3+alpha} 2 q |Phi|^2 chi + a^{1+alpha} L[chi],
 * with two Gauss laws: the SU(2) one of section 6 and
 *   (1/dx) sum_i [piA_i(n) - piA_i(n-i)] = (2 eA/kappa) Im[Phi^dag pi].
 * eA = 0 switches the U(1) sector off, chi = 0 the singlet. */
typedef struct {
    int64_t N;
    double dx, alpha, fmp2, lam, v2, g, kappa;
    int32_t pot, p;
    double eA, q;
    int32_t chi, pad;
} orc_su2u1_model;

static orc_su2_model su2_part(const orc_su2u1_model* m) {
    orc_su2_model s;
    s.N = m->N; s.dx = m->dx; s.alpha = m->alpha; s.fmp2 = m->fmp2; s.lam = m->lam; s.v2 = m->v2;
    s.g = m->g; s.kappa = m->kappa; s.pot = m->pot; s.p = m->p;
    return s;
}

/* W_i Phi(m) = e^{-i t} (U Phi(m)) with U the quaternion q */
static void whop(const double* q, double t, const double* f, double* o) {
    double u[4];
    umul(q, f, u);
    const double c = cos(t), s = sin(t);
    o[0] = c * u[0] + s * u[1];
    o[1] = c * u[1] - s * u[0];
    o[2] = c * u[2] + s * u[3];
    o[3] = c * u[3] - s * u[2];
}

/* Im[x^dag y] for doublets */
static double im_dot(const double* x, const double* y) {
    return x[0] * y[1] - x[1] * y[0] + x[2] * y[3] - x[3] * y[2];
}

static double plaq_u1(int64_t N, const double* th, int i, int j, int64_t x, int64_t y, int64_t z) {
    const int64_t V = N * N * N, n = site(N, x, y, z);
    return th[(int64_t)i * V + n] + th[(int64_t)j * V + shift(N, x, y, z, i, 1)] -
           th[(int64_t)i * V + shift(N, x, y, z, j, 1)] - th[(int64_t)j * V + n];
}

void orc_su2u1_kernels(const orc_su2u1_model* m, const double* phi, const double* u, const double* th,
                       const double* chi, double a, double* Kp, double* KB, double* KA, double* Kc) {
    const int64_t N = m->N, V = N * N * N;
    const orc_su2_model s2 = su2_part(m);
    const double A1 = pow(a, 1.0 + m->alpha), A3 = pow(a, 3.0 + m->alpha), Am = pow(a, m->alpha - 1.0);
    const double idx2 = 1.0 / (m->dx * m->dx);
    const double cJ = m->g / (m->kappa * m->dx), cM = 2.0 / (m->g * m->dx * m->dx * m->dx);
    const int u1 = m->eA != 0.0;
#pragma omp parallel for schedule(static)
    for (int64_t z = 0; z < N; ++z)
        for (int64_t y = 0; y < N; ++y)
            for (int64_t x = 0; x < N; ++x) {
                const int64_t n = site(N, x, y, z);
                double f[4], lap[4];
                getf(phi, V, n, f);
                for (int c = 0; c < 4; ++c) lap[c] = -6.0 * f[c];
                double lchi = 0.0;
                for (int i = 0; i < 3; ++i) {
                    const int64_t np = shift(N, x, y, z, i, 1), nm = shift(N, x, y, z, i, -1);
                    double q[4], qm[4], qmc[4], fp[4], fm[4], t[4], tb[4];
                    getq(u, V, i, n, q);
                    getq(u, V, i, nm, qm);
                    qconj(qm, qmc);
                    getf(phi, V, np, fp);
                    getf(phi, V, nm, fm);
                    const double ti = u1 ? th[(int64_t)i * V + n] : 0.0;
                    const double tm = u1 ? th[(int64_t)i * V + nm] : 0.0;
                    whop(q, ti, fp, t);
                    whop(qmc, -tm, fm, tb); /* W^dag(n-i) = U^dag(n-i) e^{+i theta(n-i)} */
                    for (int c = 0; c < 4; ++c) lap[c] += t[c] + tb[c];
                    double js[3];
                    im_sigma(f, t, js);
                    double mag[3] = {0, 0, 0};
                    for (int j = 0; j < 3; ++j) {
                        if (j == i) continue;
                        double P1[4], P2[4], Uj[4], Ujc[4], s1[4], Q[4];
                        plaquette(&s2, u, i, j, x, y, z, P1);
                        int64_t cm[3] = {x, y, z};
                        cm[j] = wrap(cm[j] - 1, N);
                        plaquette(&s2, u, i, j, cm[0], cm[1], cm[2], P2);
                        getq(u, V, j, site(N, cm[0], cm[1], cm[2]), Uj);
                        qconj(Uj, Ujc);
                        qmul(Ujc, P2, s1);
                        qmul(s1, Uj, Q);
                        for (int c = 0; c < 3; ++c) mag[c] += P1[c + 1] - Q[c + 1];
                    }
                    for (int c = 0; c < 3; ++c) KB[((int64_t)i * 3 + c) * V + n] = A1 * cJ * js[c] + Am * cM * mag[c];
                    if (u1) {
                        double magA = 0.0;
                        for (int j = 0; j < 3; ++j) {
                            if (j == i) continue;
                            int64_t cm[3] = {x, y, z};
                            cm[j] = wrap(cm[j] - 1, N);
                            /* Im V_ij = -sin(theta_ij) */
                            magA += -sin(plaq_u1(N, th, i, j, x, y, z)) + sin(plaq_u1(N, th, i, j, cm[0], cm[1], cm[2]));
                        }
                        KA[(int64_t)i * V + n] = A1 * 2.0 * m->eA / (m->kappa * m->dx) * im_dot(f, t) +
                                                 Am / (m->eA * m->dx * m->dx * m->dx) * magA;
                    }
                    if (m->chi) lchi += chi[np] + chi[nm];
                }
                const double mod2 = f[0] * f[0] + f[1] * f[1] + f[2] * f[2] + f[3] * f[3];
                double dv;
                gauge_potential(m->pot, m->p, m->lam, m->v2, mod2, &dv);
                const double c2 = m->chi ? chi[n] * chi[n] : 0.0;
                for (int c = 0; c < 4; ++c) Kp[(int64_t)c * V + n] = -A3 * (dv + m->q * c2) * f[c] + A1 * lap[c] * idx2;
                if (m->chi)
                    Kc[n] = -A3 * 2.0 * m->q * mod2 * chi[n] + A1 * (lchi - 6.0 * chi[n]) * idx2;
            }
}

/* out[0..8] = E_K^Phi, E_G^Phi, E_V (potential + interaction), E_K^B, E_G^B,
 * E_K^A, E_G^A, E_K^chi = <pchi^2>/(2a^6), E_G^chi = sum_i <(D_i^+ chi)^2>/(2a^2). */
void orc_su2u1_energies(const orc_su2u1_model* m, const double* phi, const double* pi, const double* u,
                        const double* piB, const double* th, const double* piA, const double* chi,
                        const double* pchi, double a, double* out) {
    const int64_t N = m->N, V = N * N * N;
    const int u1 = m->eA != 0.0;
    const orc_su2_model s2 = su2_part(m);
    double sk = 0, sg = 0, sv = 0, skb = 0, sgb = 0, ska = 0, sga = 0, skc = 0, sgc = 0;
#pragma omp parallel for reduction(+ : sk, sg, sv, skb, sgb, ska, sga, skc, sgc) schedule(static)
    for (int64_t z = 0; z < N; ++z)
        for (int64_t y = 0; y < N; ++y)
            for (int64_t x = 0; x < N; ++x) {
                const int64_t n = site(N, x, y, z);
                double f[4], p[4];
                getf(phi, V, n, f);
                getf(pi, V, n, p);
                for (int c = 0; c < 4; ++c) sk += p[c] * p[c];
                const double mod2 = f[0] * f[0] + f[1] * f[1] + f[2] * f[2] + f[3] * f[3];
                double dv;
                sv += gauge_potential(m->pot, m->p, m->lam, m->v2, mod2, &dv);
                if (m->chi) {
                    sv += m->q * mod2 * chi[n] * chi[n];
                    skc += pchi[n] * pchi[n];
                }
                for (int i = 0; i < 3; ++i) {
                    const int64_t np = shift(N, x, y, z, i, 1);
                    double q[4], fp[4], t[4];
                    getq(u, V, i, n, q);
                    getf(phi, V, np, fp);
                    whop(q, u1 ? th[(int64_t)i * V + n] : 0.0, fp, t);
                    for (int c = 0; c < 4; ++c) sg += (t[c] - f[c]) * (t[c] - f[c]);
                    for (int c = 0; c < 3; ++c) skb += piB[((int64_t)i * 3 + c) * V + n] * piB[((int64_t)i * 3 + c) * V + n];
                    if (u1) ska += piA[(int64_t)i * V + n] * piA[(int64_t)i * V + n];
                    if (m->chi) sgc += (chi[np] - chi[n]) * (chi[np] - chi[n]);
                    for (int j = i + 1; j < 3; ++j) {
                        double P[4];
                        plaquette(&s2, u, i, j, x, y, z, P);
                        sgb += 2.0 - 2.0 * P[0];
                        if (u1) sga += 1.0 - cos(plaq_u1(N, th, i, j, x, y, z));
                    }
                }
            }
    const double a2 = a * a, a4 = a2 * a2, a6 = a4 * a2, dx2 = m->dx * m->dx, dx4 = dx2 * dx2;
    out[0] = sk / V / a6;
    out[1] = sg / V / dx2 / a2;
    out[2] = sv / V;
    out[3] = m->kappa * skb / V / (2.0 * a4);
    out[4] = 2.0 * m->kappa * sgb / V / (a4 * dx4 * m->g * m->g);
    out[5] = u1 ? m->kappa * ska / V / (2.0 * a4) : 0.0;
    out[6] = u1 ? m->kappa * sga / V / (a4 * dx4 * m->eA * m->eA) : 0.0;
    out[7] = skc / V / (2.0 * a6);
    out[8] = sgc / V / dx2 / (2.0 * a2);
}

/* K_a of section 4 with every scalar (Phi, chi) weighted as a scalar and every
 * gauge energy with (alpha - 1). */
double orc_su2u1_Ka(const orc_su2u1_model* m, double a, const double* E) {
    return m->fmp2 / 3.0 * pow(a, 2.0 * m->alpha + 1.0) *
           ((m->alpha - 2.0) * (E[0] + E[7]) + m->alpha * (E[1] + E[8]) + (m->alpha + 1.0) * E[2] +
            (m->alpha - 1.0) * (E[3] + E[4] + E[5] + E[6]));
}

/* Gauss residuals: out[0..2] the SU(2) law (as orc_su2_gauss, the electric
 * momenta transported with U only: the phase drops out of the adjoint action),
 * out[3..5] = {<G^2>, <lhs^2>, <rhs^2>} of the U(1) law. */
void orc_su2u1_gauss(const orc_su2u1_model* m, const double* phi, const double* pi, const double* u,
                     const double* piB, const double* piA, double* out) {
    const orc_su2_model s2 = su2_part(m);
    orc_su2_gauss(&s2, phi, pi, u, piB, out);
    out[3] = out[4] = out[5] = 0.0;
    if (m->eA == 0.0) return;
    const int64_t N = m->N, V = N * N * N;
    double g2 = 0, l2 = 0, r2 = 0;
#pragma omp parallel for reduction(+ : g2, l2, r2) schedule(static)
    for (int64_t z = 0; z < N; ++z)
        for (int64_t y = 0; y < N; ++y)
            for (int64_t x = 0; x < N; ++x) {
                const int64_t n = site(N, x, y, z);
                double div = 0.0;
                for (int i = 0; i < 3; ++i)
                    div += (piA[(int64_t)i * V + n] - piA[(int64_t)i * V + shift(N, x, y, z, i, -1)]) / m->dx;
                double f[4], p[4];
                getf(phi, V, n, f);
                getf(pi, V, n, p);
                const double r = 2.0 * m->eA / m->kappa * im_dot(f, p);
                g2 += (div - r) * (div - r);
                l2 += div * div;
                r2 += r * r;
            }
    out[3] = g2 / V;
    out[4] = l2 / V;
    out[5] = r2 / V;
}

/* One VVn step of the combined model, the structure of orc_su2_vv_step with
 * the U(1) links drifted by the exact phase (theta += eA dx h a_1/2^{alpha-1} piA)
 * and chi drifted like Phi. */
void orc_su2u1_vv_step(const orc_su2u1_model* m, int s, const double* w, double dt, double* phi, double* pi,
                       double* u, double* piB, double* th, double* piA, double* chi, double* pchi, double* a,
                       double* b) {
    const int64_t V = m->N * m->N * m->N;
    const int u1 = m->eA != 0.0;
    const orc_su2_model s2 = su2_part(m);
    double* Kp = (double*)malloc(sizeof(double) * (size_t)(4 * V));
    double* KB = (double*)malloc(sizeof(double) * (size_t)(9 * V));
    double* KA = (double*)malloc(sizeof(double) * (size_t)(3 * V));
    double* Kc = (double*)malloc(sizeof(double) * (size_t)V);
    double E[9];
    orc_su2u1_energies(m, phi, pi, u, piB, th, piA, chi, pchi, *a, E);
    for (int p = 0; p < s; ++p) {
        const double h = w[p] * dt;
        for (int half = 0; half < 2; ++half) {
            if (half == 1) {
                const double bh = *b + 0.5 * h * orc_su2u1_Ka(m, *a, E);
                const double an = *a + h * bh, ah = 0.5 * (*a + an);
                const double cphi = h * pow(ah, -(3.0 - m->alpha));
                su2_drift(&s2, phi, pi, u, piB, cphi, m->g * m->dx * h * pow(ah, -(1.0 - m->alpha)));
                if (u1) {
                    const double cth = m->eA * m->dx * h * pow(ah, -(1.0 - m->alpha));
                    for (int64_t n = 0; n < 3 * V; ++n) th[n] += cth * piA[n];
                }
                if (m->chi)
                    for (int64_t n = 0; n < V; ++n) chi[n] += cphi * pchi[n];
                *a = an;
                *b = bh;
            }
            orc_su2u1_kernels(m, phi, u, th, chi, *a, Kp, KB, KA, Kc);
            for (int64_t n = 0; n < 4 * V; ++n) pi[n] += 0.5 * h * Kp[n];
            for (int64_t n = 0; n < 9 * V; ++n) piB[n] += 0.5 * h * KB[n];
            if (u1)
                for (int64_t n = 0; n < 3 * V; ++n) piA[n] += 0.5 * h * KA[n];
            if (m->chi)
                for (int64_t n = 0; n < V; ++n) pchi[n] += 0.5 * h * Kc[n];
        }
        orc_su2u1_energies(m, phi, pi, u, piB, th, piA, chi, pchi, *a, E);
        *b += 0.5 * h * orc_su2u1_Ka(m, *a, E);
    }
    free(Kp);
    free(KB);
    free(KA);
    free(Kc);
}

/* ------------------------------------------------ Gauss-Legendre (implicit RK) */

/* One step of the s-stage Gauss-Legendre implicit Runge-Kutta method of
 * sections 3.4.2 and 4.3.3 in Scheme II (Hamiltonian variables):
 *   y = (phi, pi, a, b),  F(y) = (a^{-(3-alpha)} pi, K[a, phi], b, K_a[a, E(y)]),
 *   Y^(l) = y(n0) + dt sum_m A_lm D^(m),  D^(l) = F(Y^(l)),
 *   y(n0 + 1) = y(n0) + dt sum_m c_m D^(m),
 * with the Butcher tableau (A, c) of order 2s.  The stage equations are solved
 * by Jacobi fixed-point iteration from D = 0 (the first sweep gives F(y(n0))
 * for every stage) until ||D_new - D_old||_2 <= tol ||D_new||_2 over all
 * fields, stages and the two scalars, or maxit sweeps.  Returns the sweeps. */
int orc_scalar_gl_step(const orc_scalar_model* m, int s, const double* A, const double* c, double dt, double tol,
                       int maxit, double* phi, double* pi, double* a, double* b) {
    const int64_t V = m->N * m->N * m->N, M = (int64_t)m->Ns * V;
    double* D0 = (double*)calloc((size_t)(2 * s * M), sizeof(double)); /* stage l: dphi at 2lM, dpi at (2l+1)M */
    double* D1 = (double*)calloc((size_t)(2 * s * M), sizeof(double));
    double* ps = (double*)malloc(sizeof(double) * (size_t)M);
    double* qs = (double*)malloc(sizeof(double) * (size_t)M);
    double Da0[5] = {0}, Db0[5] = {0}, Da1[5] = {0}, Db1[5] = {0};
    double* Dold = D0;
    double* Dnew = D1;
    double *Daold = Da0, *Dbold = Db0, *Danew = Da1, *Dbnew = Db1;
    int it = 0;
    for (it = 1; it <= maxit; ++it) {
        double dd = 0.0, nn = 0.0;
        for (int l = 0; l < s; ++l) {
            double al = *a, bl = *b;
            for (int mm = 0; mm < s; ++mm) {
                al += dt * A[l * s + mm] * Daold[mm];
                bl += dt * A[l * s + mm] * Dbold[mm];
            }
            for (int64_t n = 0; n < M; ++n) {
                double x = phi[n], y = pi[n];
                for (int mm = 0; mm < s; ++mm) {
                    x += dt * A[l * s + mm] * Dold[(int64_t)(2 * mm) * M + n];
                    y += dt * A[l * s + mm] * Dold[(int64_t)(2 * mm + 1) * M + n];
                }
                ps[n] = x;
                qs[n] = y;
            }
            double* dphi = Dnew + (int64_t)(2 * l) * M;
            double* dpi = Dnew + (int64_t)(2 * l + 1) * M;
            orc_scalar_kernel(m, ps, al, dpi);
            const double cdr = pow(al, -(3.0 - m->alpha));
            for (int64_t n = 0; n < M; ++n) dphi[n] = cdr * qs[n];
            double E[6];
            orc_scalar_energies(m, ps, qs, al, E);
            Danew[l] = bl;
            Dbnew[l] = orc_scalar_Ka(m, al, E);
            for (int64_t n = 0; n < M; ++n) {
                const double e1 = dphi[n] - Dold[(int64_t)(2 * l) * M + n], e2 = dpi[n] - Dold[(int64_t)(2 * l + 1) * M + n];
                dd += e1 * e1 + e2 * e2;
                nn += dphi[n] * dphi[n] + dpi[n] * dpi[n];
            }
            dd += (Danew[l] - Daold[l]) * (Danew[l] - Daold[l]) + (Dbnew[l] - Dbold[l]) * (Dbnew[l] - Dbold[l]);
            nn += Danew[l] * Danew[l] + Dbnew[l] * Dbnew[l];
        }
        double* t = Dold; Dold = Dnew; Dnew = t;
        t = Daold; Daold = Danew; Danew = t;
        t = Dbold; Dbold = Dbnew; Dbnew = t;
        if (dd <= tol * tol * nn) break;
    }
    for (int64_t n = 0; n < M; ++n)
        for (int mm = 0; mm < s; ++mm) {
            phi[n] += dt * c[mm] * Dold[(int64_t)(2 * mm) * M + n];
            pi[n] += dt * c[mm] * Dold[(int64_t)(2 * mm + 1) * M + n];
        }
    double da = 0.0, db = 0.0;
    for (int mm = 0; mm < s; ++mm) {
        da += dt * c[mm] * Daold[mm];
        db += dt * c[mm] * Dbold[mm];
    }
    *a += da;
    *b += db;
    free(D0); free(D1); free(ps); free(qs);
    return it > maxit ? maxit : it;
}

/* Threads of the OpenMP loops above (the benchmark's CPU leg times the oracle
 * on one thread and on all cores); without OpenMP both are no-ops on 1. */
void orc_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}
int orc_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
