/*
 * colatus_oracle.c -- FP64 CPU oracle for the all-pairs comoving gravity path
 * of COLATUS (Stalder et al., arXiv 1208.3444).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load this library.  It shares no code,
 * header or constant with the CUDA library and must never be reached from the
 * product path.
 *
 * Everything here is plain double-precision loops written straight from the
 * paper's equations; nothing is blocked, fused or reordered beyond what the
 * definition states.  Parallel loops (OpenMP) only split independent target
 * rows; each row is summed sequentially over j = 0..N-1.
 *
 * Sign convention (reading of Eq. 1): the printed right-hand side of Eq. 1,
 * a^-3 G sum m_j (x_k - x_j)/s^3, points AWAY from the other bodies; Eq. 6
 * and gravity itself want the attractive field, so the raw force used here is
 *
 *     F_k = G * sum_{j != k} m_j (x_j - x_k) / (|x_j - x_k|^2 + eps^2)^{3/2}
 *
 * and the comoving acceleration is a^-3 F_k.  The a^-3 factor is applied by
 * the caller (integrator), once.
 *
 * Layout: positions x[3*N] (x0,y0,z0,x1,...), masses m[N], all double.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>

/* Raw force F (Eq. 1, attractive reading) summed over unordered pairs j<k.
 * Each pair is evaluated once and applied to both bodies with opposite sign,
 * so m_k F_kj = -m_j F_jk holds bit for bit (Newton's third law). */
void colatus_oracle_forces_pairwise(int64_t n, const double *x, const double *m,
                                    double eps, double G, double *acc)
{
    const double eps2 = eps * eps;
    for (int64_t k = 0; k < 3 * n; ++k) acc[k] = 0.0;
    for (int64_t k = 0; k < n; ++k) {
        for (int64_t j = k + 1; j < n; ++j) {
            double dx = x[3 * j + 0] - x[3 * k + 0];
            double dy = x[3 * j + 1] - x[3 * k + 1];
            double dz = x[3 * j + 2] - x[3 * k + 2];
            double s2 = dx * dx + dy * dy + dz * dz + eps2;
            double inv3 = 1.0 / (s2 * sqrt(s2));
            /* pull on k toward j, on j toward k */
            double qk = G * m[j] * inv3;
            double qj = G * m[k] * inv3;
            acc[3 * k + 0] += qk * dx;
            acc[3 * k + 1] += qk * dy;
            acc[3 * k + 2] += qk * dz;
            acc[3 * j + 0] -= qj * dx;
            acc[3 * j + 1] -= qj * dy;
            acc[3 * j + 2] -= qj * dz;
        }
    }
}

/* Raw force F for a subset of target rows against all N sources, summed
 * row by row in source order; the self pair is skipped as in the paper's
 * Appendix A kernel (idx != i).  out[3*r] is the force on body rows[r]. */
void colatus_oracle_forces_rows(int64_t n, const double *x, const double *m,
                                double eps, double G, const int64_t *rows,
                                int64_t nrows, double *out)
{
    const double eps2 = eps * eps;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t r = 0; r < nrows; ++r) {
        const int64_t k = rows[r];
        double ax = 0.0, ay = 0.0, az = 0.0;
        for (int64_t j = 0; j < n; ++j) {
            if (j == k) continue;
            double dx = x[3 * j + 0] - x[3 * k + 0];
            double dy = x[3 * j + 1] - x[3 * k + 1];
            double dz = x[3 * j + 2] - x[3 * k + 2];
            double s2 = dx * dx + dy * dy + dz * dz + eps2;
            double w = m[j] / (s2 * sqrt(s2));
            ax += w * dx;
            ay += w * dy;
            az += w * dz;
        }
        out[3 * r + 0] = G * ax;
        out[3 * r + 1] = G * ay;
        out[3 * r + 2] = G * az;
    }
}

/* Softened potential phi_k = -G sum_{j != k} m_j / s_kj, the potential whose
 * negative gradient (times m_k) is the attractive force above.  Used for the
 * potential energy W_x = (1/2) sum_k m_k phi_k. */
void colatus_oracle_potential_rows(int64_t n, const double *x, const double *m,
                                   double eps, double G, const int64_t *rows,
                                   int64_t nrows, double *phi)
{
    const double eps2 = eps * eps;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t r = 0; r < nrows; ++r) {
        const int64_t k = rows[r];
        double s = 0.0;
        for (int64_t j = 0; j < n; ++j) {
            if (j == k) continue;
            double dx = x[3 * j + 0] - x[3 * k + 0];
            double dy = x[3 * j + 1] - x[3 * k + 1];
            double dz = x[3 * j + 2] - x[3 * k + 2];
            double s2 = dx * dx + dy * dy + dz * dz + eps2;
            s += m[j] / sqrt(s2);
        }
        phi[r] = -G * s;
    }
}

/* Vector-Jacobian product of the raw force F(x, m) with a co-vector lam[3N]:
 *   L = sum_k lam_k . F_k
 *   gx_q = dL/dx_q = G sum_{j != q} J(d_qj) (m_q lam_j - m_j lam_q)
 *   gm_q = dL/dm_q = G sum_{k != q} lam_k . (x_q - x_k) / s_kq^3
 * with d_qj = x_j - x_q, s^2 = |d|^2 + eps^2 and J(d) = I/s^3 - 3 d d^T / s^5
 * (the Jacobian of d/s^3 with respect to d).  Derived by differentiating the
 * Eq. 1 sum; J is even in d, which is what makes both terms share J(d_qj). */
void colatus_oracle_vjp_rows(int64_t n, const double *x, const double *m,
                             const double *lam, double eps, double G,
                             const int64_t *rows, int64_t nrows,
                             double *gx, double *gm)
{
    const double eps2 = eps * eps;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t r = 0; r < nrows; ++r) {
        const int64_t q = rows[r];
        double g0 = 0.0, g1 = 0.0, g2 = 0.0, h = 0.0;
        for (int64_t j = 0; j < n; ++j) {
            if (j == q) continue;
            double d0 = x[3 * j + 0] - x[3 * q + 0];
            double d1 = x[3 * j + 1] - x[3 * q + 1];
            double d2 = x[3 * j + 2] - x[3 * q + 2];
            double s2 = d0 * d0 + d1 * d1 + d2 * d2 + eps2;
            double inv3 = 1.0 / (s2 * sqrt(s2));
            double inv5 = inv3 / s2;
            double w0 = m[q] * lam[3 * j + 0] - m[j] * lam[3 * q + 0];
            double w1 = m[q] * lam[3 * j + 1] - m[j] * lam[3 * q + 1];
            double w2 = m[q] * lam[3 * j + 2] - m[j] * lam[3 * q + 2];
            double dw = d0 * w0 + d1 * w1 + d2 * w2;
            g0 += w0 * inv3 - 3.0 * d0 * dw * inv5;
            g1 += w1 * inv3 - 3.0 * d1 * dw * inv5;
            g2 += w2 * inv3 - 3.0 * d2 * dw * inv5;
            /* x_q - x_j = -d_qj */
            h += -(lam[3 * j + 0] * d0 + lam[3 * j + 1] * d1 + lam[3 * j + 2] * d2) * inv3;
        }
        gx[3 * r + 0] = G * g0;
        gx[3 * r + 1] = G * g1;
        gx[3 * r + 2] = G * g2;
        gm[r] = G * h;
    }
}

/* Jacobian-vector (tangent) product of the raw force with a perturbation
 * (dx[3N], dm[N]); dm may be NULL (no mass perturbation):
 *   dF_k = G sum_{j != k} [ m_j J(d_kj) (dx_j - dx_k) + dm_j d_kj / s_kj^3 ]. */
void colatus_oracle_jvp_rows(int64_t n, const double *x, const double *m,
                             const double *dx, const double *dm, double eps,
                             double G, const int64_t *rows, int64_t nrows,
                             double *df)
{
    const double eps2 = eps * eps;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t r = 0; r < nrows; ++r) {
        const int64_t k = rows[r];
        double f0 = 0.0, f1 = 0.0, f2 = 0.0;
        for (int64_t j = 0; j < n; ++j) {
            if (j == k) continue;
            double d0 = x[3 * j + 0] - x[3 * k + 0];
            double d1 = x[3 * j + 1] - x[3 * k + 1];
            double d2 = x[3 * j + 2] - x[3 * k + 2];
            double s2 = d0 * d0 + d1 * d1 + d2 * d2 + eps2;
            double inv3 = 1.0 / (s2 * sqrt(s2));
            double inv5 = inv3 / s2;
            double u0 = dx[3 * j + 0] - dx[3 * k + 0];
            double u1 = dx[3 * j + 1] - dx[3 * k + 1];
            double u2 = dx[3 * j + 2] - dx[3 * k + 2];
            double du = d0 * u0 + d1 * u1 + d2 * u2;
            f0 += m[j] * (u0 * inv3 - 3.0 * d0 * du * inv5);
            f1 += m[j] * (u1 * inv3 - 3.0 * d1 * du * inv5);
            f2 += m[j] * (u2 * inv3 - 3.0 * d2 * du * inv5);
            if (dm) {
                f0 += dm[j] * d0 * inv3;
                f1 += dm[j] * d1 * inv3;
                f2 += dm[j] * d2 * inv3;
            }
        }
        df[3 * r + 0] = G * f0;
        df[3 * r + 1] = G * f1;
        df[3 * r + 2] = G * f2;
    }
}

/* Periodic boundaries (Sec. II: periodic, for a homogeneous distribution):
 * the real-space part of the Ewald sum of the Newtonian pull over all images
 * x_j + n L (n integer, |n_c| <= nreal around the minimum image), plus the
 * softening correction of the nearest image, for target rows:
 *
 *   out_k = G sum_j m_j [ sum_n N_S(d_j + n L) + P(d_j) - N(d_j) ]
 *
 * d_j = minimum image of x_j - x_k, N(d) = d/|d|^3, P(d) = d/(|d|^2+eps^2)^1.5,
 * N_S(r) = r [erfc(alpha |r|)/|r|^3 + 2 alpha/sqrt(pi) exp(-alpha^2 |r|^2)/|r|^2],
 * and every |r| = 0 term (the self pair's own cell) left out.  The
 * reciprocal-space part is added by the caller.  Brute force: one loop per
 * image, in order. */
void colatus_oracle_ewald_real_rows(int64_t n, const double *x, const double *m,
                                    double eps, double G, double L, double alpha,
                                    int64_t nreal, const int64_t *rows, int64_t nrows,
                                    double *out)
{
    const double eps2 = eps * eps;
    const double c_g = 2.0 * alpha / sqrt(acos(-1.0));   /* 2 alpha / sqrt(pi) */
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t r = 0; r < nrows; ++r) {
        const int64_t k = rows[r];
        double ax = 0.0, ay = 0.0, az = 0.0;
        for (int64_t j = 0; j < n; ++j) {
            double d[3];
            for (int c = 0; c < 3; ++c) {
                d[c] = x[3 * j + c] - x[3 * k + c];
                d[c] -= L * nearbyint(d[c] / L);
            }
            const double d2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
            if (d2 > 0.0) {
                /* nearest image: Plummer instead of Newton */
                const double s2 = d2 + eps2;
                const double w = m[j] * (1.0 / (s2 * sqrt(s2)) - 1.0 / (d2 * sqrt(d2)));
                ax += w * d[0];
                ay += w * d[1];
                az += w * d[2];
            }
            for (int64_t i0 = -nreal; i0 <= nreal; ++i0)
                for (int64_t i1 = -nreal; i1 <= nreal; ++i1)
                    for (int64_t i2 = -nreal; i2 <= nreal; ++i2) {
                        const double e0 = d[0] + L * (double)i0;
                        const double e1 = d[1] + L * (double)i1;
                        const double e2 = d[2] + L * (double)i2;
                        const double q2 = e0 * e0 + e1 * e1 + e2 * e2;
                        if (q2 == 0.0) continue;
                        const double q = sqrt(q2);
                        const double w = m[j] * (erfc(alpha * q) / (q2 * q) +
                                                 c_g * exp(-alpha * alpha * q2) / q2);
                        ax += w * e0;
                        ay += w * e1;
                        az += w * e2;
                    }
        }
        out[3 * r + 0] = G * ax;
        out[3 * r + 1] = G * ay;
        out[3 * r + 2] = G * az;
    }
}

/* Jacobian of the real-space periodic pair term of
 * colatus_oracle_ewald_real_rows with respect to the separation d (the
 * minimum image of x_j - x_k): the pair term is R(d) = sum_n N_S(d + n L)
 * + P(d) - N(d), so, differentiating each term (Sec. II periodic boundaries,
 * Ewald split; J is symmetric and even in d):
 *   N_S(e) = e h(q):       J = h I + (h'(q)/q) e e^T,
 *       h = erfc(alpha q)/q^3 + c_g exp(-alpha^2 q^2)/q^2,
 *       h'(q)/q = -3 h/q^2 - 2 alpha^2 c_g exp(-alpha^2 q^2)/q^2;
 *   P(d) = d/s^3:          J = I/s^3 - 3 d d^T/s^5,  s^2 = |d|^2 + eps^2;
 *   N(d) = d/|d|^3:        J = I/r^3 - 3 d d^T/r^5.
 * Every q = 0 image is left out, as in the force.  At d = 0 exactly (two
 * distinct bodies at one point) the nearest image's P - N + N_S is taken at
 * its limit, (1/eps^3 - (4/3) alpha^3/sqrt(pi)) I.  Also returns R(d) in Rv. */
static void ewald_real_pair_jacobian(const double d[3], double eps2, double L, double alpha,
                                     int64_t nreal, double J[3][3], double Rv[3])
{
    const double pi = acos(-1.0);
    const double c_g = 2.0 * alpha / sqrt(pi);
    for (int a = 0; a < 3; ++a) {
        Rv[a] = 0.0;
        for (int b = 0; b < 3; ++b) J[a][b] = 0.0;
    }
    const double d2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    if (d2 > 0.0) {
        const double s2 = d2 + eps2, s = sqrt(s2), r = sqrt(d2);
        const double is3 = 1.0 / (s2 * s), is5 = is3 / s2;
        const double ir3 = 1.0 / (d2 * r), ir5 = ir3 / d2;
        for (int a = 0; a < 3; ++a) {
            Rv[a] += (is3 - ir3) * d[a];
            J[a][a] += is3 - ir3;
            for (int b = 0; b < 3; ++b) J[a][b] += -3.0 * (is5 - ir5) * d[a] * d[b];
        }
    } else {
        const double lim = 1.0 / (eps2 * sqrt(eps2)) - 4.0 / 3.0 * alpha * alpha * alpha / sqrt(pi);
        for (int a = 0; a < 3; ++a) J[a][a] += lim;
    }
    for (int64_t i0 = -nreal; i0 <= nreal; ++i0)
        for (int64_t i1 = -nreal; i1 <= nreal; ++i1)
            for (int64_t i2 = -nreal; i2 <= nreal; ++i2) {
                const double e[3] = {d[0] + L * (double)i0, d[1] + L * (double)i1,
                                     d[2] + L * (double)i2};
                const double q2 = e[0] * e[0] + e[1] * e[1] + e[2] * e[2];
                if (q2 == 0.0) continue;
                const double q = sqrt(q2);
                const double g = exp(-alpha * alpha * q2);
                const double h = erfc(alpha * q) / (q2 * q) + c_g * g / q2;
                const double hq = -3.0 * h / q2 - 2.0 * alpha * alpha * c_g * g / q2;
                for (int a = 0; a < 3; ++a) {
                    Rv[a] += h * e[a];
                    J[a][a] += h;
                    for (int b = 0; b < 3; ++b) J[a][b] += hq * e[a] * e[b];
                }
            }
}

static void min_image(const double *x, int64_t j, int64_t k, double L, double d[3])
{
    for (int c = 0; c < 3; ++c) {
        d[c] = x[3 * j + c] - x[3 * k + c];
        d[c] -= L * nearbyint(d[c] / L);
    }
}

/* Real-space part of the periodic force's directional derivative along
 * (dx, dm) (dm may be NULL), for target rows k:
 *   out_k = G sum_{j != k} [ m_j J_R(d_kj) (dx_j - dx_k) + dm_j R(d_kj) ]. */
void colatus_oracle_ewald_real_jvp_rows(int64_t n, const double *x, const double *m,
                                        const double *dx, const double *dm, double eps, double G,
                                        double L, double alpha, int64_t nreal,
                                        const int64_t *rows, int64_t nrows, double *out)
{
    const double eps2 = eps * eps;
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t r = 0; r < nrows; ++r) {
        const int64_t k = rows[r];
        double acc[3] = {0.0, 0.0, 0.0};
        for (int64_t j = 0; j < n; ++j) {
            if (j == k) continue;
            double d[3], J[3][3], Rv[3];
            min_image(x, j, k, L, d);
            ewald_real_pair_jacobian(d, eps2, L, alpha, nreal, J, Rv);
            const double u[3] = {dx[3 * j] - dx[3 * k], dx[3 * j + 1] - dx[3 * k + 1],
                                 dx[3 * j + 2] - dx[3 * k + 2]};
            for (int a = 0; a < 3; ++a) {
                acc[a] += m[j] * (J[a][0] * u[0] + J[a][1] * u[1] + J[a][2] * u[2]);
                if (dm) acc[a] += dm[j] * Rv[a];
            }
        }
        for (int a = 0; a < 3; ++a) out[3 * r + a] = G * acc[a];
    }
}

/* Real-space part of the periodic force's vector-Jacobian product: for
 * L = sum_k lam_k . F_k and target rows i,
 *   gx_i = G sum_{j != i} J_R(d_ij) (m_i lam_j - m_j lam_i),
 *   gm_i = -G sum_{j != i} lam_j . R(d_ij). */
void colatus_oracle_ewald_real_vjp_rows(int64_t n, const double *x, const double *m,
                                        const double *lam, double eps, double G, double L,
                                        double alpha, int64_t nreal, const int64_t *rows,
                                        int64_t nrows, double *gx, double *gm)
{
    const double eps2 = eps * eps;
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t r = 0; r < nrows; ++r) {
        const int64_t i = rows[r];
        double acc[3] = {0.0, 0.0, 0.0}, am = 0.0;
        for (int64_t j = 0; j < n; ++j) {
            if (j == i) continue;
            double d[3], J[3][3], Rv[3];
            min_image(x, j, i, L, d);
            ewald_real_pair_jacobian(d, eps2, L, alpha, nreal, J, Rv);
            double u[3];
            for (int a = 0; a < 3; ++a) u[a] = m[i] * lam[3 * j + a] - m[j] * lam[3 * i + a];
            for (int a = 0; a < 3; ++a)
                acc[a] += J[a][0] * u[0] + J[a][1] * u[1] + J[a][2] * u[2];
            am += lam[3 * j] * Rv[0] + lam[3 * j + 1] * Rv[1] + lam[3 * j + 2] * Rv[2];
        }
        for (int a = 0; a < 3; ++a) gx[3 * r + a] = G * acc[a];
        gm[r] = -G * am;
    }
}

/* Number of OpenMP threads the parallel loops above use. */
int colatus_oracle_threads(void)
{
    int t = 1;
#pragma omp parallel
    {
#pragma omp single
        {
#ifdef _OPENMP
            extern int omp_get_num_threads(void);
            t = omp_get_num_threads();
#endif
        }
    }
    return t;
}

/* Run the parallel loops above on n threads from now on (n >= 1; the
 * OpenMP default otherwise).  Used to time the oracle on one core. */
void colatus_oracle_set_threads(int n)
{
#ifdef _OPENMP
    extern void omp_set_num_threads(int);
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}
