/*
 * ssm_oracle.c -- plain, slow FP64 CPU oracle for the simplified string method of
 * Heistracher et al., "GPU-accelerated atomistic energy barrier calculations of skyrmion
 * annihilations" (arXiv:1804.07135).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the benchmark's CPU-baseline leg
 * may load this library.  It shares no code, header or table with the CUDA path; the two meet only
 * through the seeded inputs that the tests hand to both.
 *
 * Reduced units (stated once, used everywhere below):
 *   - energies are in units of the exchange constant J's unit; lengths in lattice constants a;
 *   - spins are the unit vectors s_i (the paper's \hat s_i);
 *   - the field is h_i = -dE/ds_i, i.e. mu0 |S| H_eff of Eq. 2 with mu0|S| absorbed;
 *   - the dipole strength is w = mu0 |S|^2 / (4 pi a^3), so the last term of Eq. 1 reads
 *     -w sum_{i<j} [3 (s_i.r)(s_j.r) - s_i.s_j] / r^3 with r in lattice units.
 * Lattice: simple cubic, nx*ny*nz sites, open (free) boundaries (Sec. II).  Site index
 * i = (z*ny + y)*nx + x; spin arrays are [site][3] (x,y,z components); a string is [image][site][3].
 *
 * Parity status: every function here is pinned by a CPU test against closed forms, finite
 * differences, geometry or an independent library routine, except the barrier value of a general
 * string run (or_string_run and its variants on a workload whose saddle has no closed form), whose
 * only check beyond the pinned parts it is composed of is sanity (barrier >= 0): "parity unpinned" for
 * that number.  With the climbing image the barrier is pinned where the saddle is known exactly (a
 * lone spin under anisotropy: K; a small ferromagnet's coherent rotation: N K).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    int nx, ny, nz;
    double J, D, K, w;
} or_model;

static int site(const or_model* m, int x, int y, int z) { return (z * m->ny + y) * m->nx + x; }

/* Eq. 7: dipole-dipole tensor D(r) = (1/4pi) (3 r r^T / r^5 - I / r^3) for r != 0, returned as its
 * six unique entries (xx, yy, zz, xy, xz, yz). */
void or_dipole_tensor(double rx, double ry, double rz, double out[6]) {
    const double r2 = rx * rx + ry * ry + rz * rz;
    const double r = sqrt(r2);
    const double r3 = r2 * r, r5 = r3 * r2;
    const double c = 1.0 / (4.0 * M_PI);
    out[0] = c * (3.0 * rx * rx / r5 - 1.0 / r3);
    out[1] = c * (3.0 * ry * ry / r5 - 1.0 / r3);
    out[2] = c * (3.0 * rz * rz / r5 - 1.0 / r3);
    out[3] = c * (3.0 * rx * ry / r5);
    out[4] = c * (3.0 * rx * rz / r5);
    out[5] = c * (3.0 * ry * rz / r5);
}

/* Eq. 1, term by term, straight from the Hamiltonian (not from the field).
 * <i,j> runs over nearest-neighbour bonds, each unordered bond once; r_ij points from i to j.
 *   exchange:  -J s_i.s_j
 *   DMI:        D (r_ij x z).(s_i x s_j)
 *   anisotropy: -K (s_i.z)^2
 *   dipole:     -w [3 (s_i.r)(s_j.r) - s_i.s_j] / r^3 over unordered pairs i<j (the paper's
 *               1/(8pi) over ordered pairs i != j is 1/(4pi) over unordered ones).
 * out = {E_exchange, E_dmi, E_anisotropy, E_dipole, E_total}. */
void or_energy_terms(const or_model* m, const double* s, double out[5]) {
    const int N = m->nx * m->ny * m->nz;
    double e_exc = 0, e_dmi = 0, e_ani = 0, e_dip = 0;
    static const int dirs[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
    for (int z = 0; z < m->nz; ++z)
        for (int y = 0; y < m->ny; ++y)
            for (int x = 0; x < m->nx; ++x) {
                const int i = site(m, x, y, z);
                const double* si = s + 3 * i;
                for (int d = 0; d < 3; ++d) {
                    const int xj = x + dirs[d][0], yj = y + dirs[d][1], zj = z + dirs[d][2];
                    if (xj >= m->nx || yj >= m->ny || zj >= m->nz) continue; /* open boundary */
                    const double* sj = s + 3 * site(m, xj, yj, zj);
                    e_exc += -m->J * (si[0] * sj[0] + si[1] * sj[1] + si[2] * sj[2]);
                    /* r_ij x z for r_ij = (rx, ry, rz): (ry, -rx, 0) */
                    const double a0 = (double)dirs[d][1], a1 = -(double)dirs[d][0], a2 = 0.0;
                    const double c0 = si[1] * sj[2] - si[2] * sj[1];
                    const double c1 = si[2] * sj[0] - si[0] * sj[2];
                    const double c2 = si[0] * sj[1] - si[1] * sj[0];
                    e_dmi += m->D * (a0 * c0 + a1 * c1 + a2 * c2);
                }
                e_ani += -m->K * si[2] * si[2];
            }
    if (m->w != 0.0) {
        for (int i = 0; i < N; ++i) {
            const int xi = i % m->nx, yi = (i / m->nx) % m->ny, zi = i / (m->nx * m->ny);
            const double* si = s + 3 * i;
            for (int j = i + 1; j < N; ++j) {
                const int xj = j % m->nx, yj = (j / m->nx) % m->ny, zj = j / (m->nx * m->ny);
                const double rx = xj - xi, ry = yj - yi, rz = zj - zi;
                const double r = sqrt(rx * rx + ry * ry + rz * rz);
                const double ux = rx / r, uy = ry / r, uz = rz / r;
                const double* sj = s + 3 * j;
                const double sir = si[0] * ux + si[1] * uy + si[2] * uz;
                const double sjr = sj[0] * ux + sj[1] * uy + sj[2] * uz;
                const double sij = si[0] * sj[0] + si[1] * sj[1] + si[2] * sj[2];
                e_dip += -m->w * (3.0 * sir * sjr - sij) / (r * r * r);
            }
        }
    }
    out[0] = e_exc;
    out[1] = e_dmi;
    out[2] = e_ani;
    out[3] = e_dip;
    out[4] = e_exc + e_dmi + e_ani + e_dip;
}

/* Table of Eq. 7 at every lattice offset (dx, dy, dz), |dx|<nx, |dy|<ny, |dz|<nz; entry 0 at the
 * origin (no self term).  Layout [dz+nz-1][dy+ny-1][dx+nx-1][6].  Caller frees. */
static double* dipole_table(const or_model* m) {
    const int Lx = 2 * m->nx - 1, Ly = 2 * m->ny - 1, Lz = 2 * m->nz - 1;
    double* t = (double*)calloc((size_t)Lx * Ly * Lz * 6, sizeof(double));
    if (!t) return NULL;
    for (int dz = -(m->nz - 1); dz <= m->nz - 1; ++dz)
        for (int dy = -(m->ny - 1); dy <= m->ny - 1; ++dy)
            for (int dx = -(m->nx - 1); dx <= m->nx - 1; ++dx) {
                if (dx == 0 && dy == 0 && dz == 0) continue;
                double* e = t + 6 * (((size_t)(dz + m->nz - 1) * Ly + (dy + m->ny - 1)) * Lx + (dx + m->nx - 1));
                or_dipole_tensor(dx, dy, dz, e);
            }
    return t;
}

/* Eqs. 2-6: the effective field h_i = -dE/ds_i at site (x, y, z) of one image.
 *   exchange   (Eq. 3): J sum over the (up to 6) nearest neighbours of s_j
 *   DMI        (Eq. 4): -D ( s_z^{i+x} - s_z^{i-x},  s_z^{i+y} - s_z^{i-y},
 *                            -s_x^{i+x} + s_x^{i-x} - s_y^{i+y} + s_y^{i-y} ), missing neighbours 0
 *   anisotropy (Eq. 5): 2 K (s_i.z) z
 *   dipole     (Eq. 6): 4 pi w sum_{j != i} D(r_ij) s_j with D of Eq. 7, summed directly (O(N)).
 * `table` is the Eq. 7 table of dipole_table() (may be NULL when w == 0). */
static void field_site(const or_model* m, const double* table, const double* s, int x, int y, int z, double* hout) {
    const int nx = m->nx, ny = m->ny, nz = m->nz, N = nx * ny * nz;
#define S(xx, yy, zz, c) \
    (((xx) < 0 || (xx) >= nx || (yy) < 0 || (yy) >= ny || (zz) < 0 || (zz) >= nz) ? 0.0 : s[3 * site(m, xx, yy, zz) + (c)])
    const int i = site(m, x, y, z);
    double hx = 0, hy = 0, hz = 0;
    /* Eq. 3 */
    for (int c = 0; c < 3; ++c) {
        const double sum = S(x + 1, y, z, c) + S(x - 1, y, z, c) + S(x, y + 1, z, c) + S(x, y - 1, z, c) +
                           S(x, y, z + 1, c) + S(x, y, z - 1, c);
        if (c == 0) hx += m->J * sum;
        if (c == 1) hy += m->J * sum;
        if (c == 2) hz += m->J * sum;
    }
    /* Eq. 4 */
    hx += -m->D * (S(x + 1, y, z, 2) - S(x - 1, y, z, 2));
    hy += -m->D * (S(x, y + 1, z, 2) - S(x, y - 1, z, 2));
    hz += -m->D * (-S(x + 1, y, z, 0) + S(x - 1, y, z, 0) - S(x, y + 1, z, 1) + S(x, y - 1, z, 1));
    /* Eq. 5 */
    hz += 2.0 * m->K * s[3 * i + 2];
#undef S
    if (m->w != 0.0 && table) {
        /* Eq. 6 */
        const int Lx = 2 * nx - 1, Ly = 2 * ny - 1;
        const double pref = 4.0 * M_PI * m->w;
        double ax = 0, ay = 0, az = 0;
        for (int j = 0; j < N; ++j) {
            if (j == i) continue;
            const int xj = j % nx, yj = (j / nx) % ny, zj = j / (nx * ny);
            const double* d = table + 6 * (((size_t)(zj - z + nz - 1) * Ly + (yj - y + ny - 1)) * Lx + (xj - x + nx - 1));
            const double* sj = s + 3 * j;
            ax += d[0] * sj[0] + d[3] * sj[1] + d[4] * sj[2];
            ay += d[3] * sj[0] + d[1] * sj[1] + d[5] * sj[2];
            az += d[4] * sj[0] + d[5] * sj[1] + d[2] * sj[2];
        }
        hx += pref * ax;
        hy += pref * ay;
        hz += pref * az;
    }
    hout[0] = hx;
    hout[1] = hy;
    hout[2] = hz;
}

static void field_one(const or_model* m, const double* table, const double* s, double* h) {
    for (int z = 0; z < m->nz; ++z)
        for (int y = 0; y < m->ny; ++y)
            for (int x = 0; x < m->nx; ++x) field_site(m, table, s, x, y, z, h + 3 * site(m, x, y, z));
}

/* Eqs. 2-7 at selected sites of one image: h_out[3*q..] = h at site index sites[q]. Returns 0, or -1
 * when out of memory or a site index is out of range. */
int or_field_at(const or_model* m, const double* s, int n_sel, const int* sites, double* h_out) {
    const int N = m->nx * m->ny * m->nz;
    for (int q = 0; q < n_sel; ++q)
        if (sites[q] < 0 || sites[q] >= N) return -1;
    double* table = NULL;
    if (m->w != 0.0) {
        table = dipole_table(m);
        if (!table) return -1;
    }
#pragma omp parallel for schedule(dynamic, 4)
    for (int q = 0; q < n_sel; ++q) {
        const int i = sites[q];
        field_site(m, table, s, i % m->nx, (i / m->nx) % m->ny, i / (m->nx * m->ny), h_out + 3 * q);
    }
    free(table);
    return 0;
}

/* Eqs. 2-6 for `n_images` images stored back to back ([image][site][3]). Returns 0, or -1 when out of memory. */
int or_field(const or_model* m, int n_images, const double* s, double* h) {
    const int N = m->nx * m->ny * m->nz;
    double* table = NULL;
    if (m->w != 0.0) {
        table = dipole_table(m);
        if (!table) return -1;
    }
#pragma omp parallel for schedule(dynamic, 1)
    for (int k = 0; k < n_images; ++k) field_one(m, table, s + (size_t)3 * N * k, h + (size_t)3 * N * k);
    free(table);
    return 0;
}

/* Only the dipole part of Eq. 6 (exchange, DMI and anisotropy left out), for one image. */
int or_dipole_field(const or_model* m, const double* s, double* h) {
    or_model d = *m;
    d.J = 0.0;
    d.D = 0.0;
    d.K = 0.0;
    return or_field(&d, 1, s, h);
}

/* Eq. 8: E = -(1/2) sum_i h_i . s_i (exact for Eq. 1, which is a homogeneous quadratic in the spins). */
double or_energy_from_field(int n_sites, const double* s, const double* h) {
    double e = 0.0;
    for (int i = 0; i < 3 * n_sites; ++i) e += h[i] * s[i];
    return -0.5 * e;
}

/* Eq. 10 with the potential force of Eq. 13 (Appendix A): one explicit step of length dt along
 * F = h - (s.h) s (the component of h perpendicular to s; the LLG prefactors are absorbed into dt),
 * followed by renormalisation to unit length, at every site. */
void or_step(int n_sites, double dt, const double* h, double* s) {
    for (int i = 0; i < n_sites; ++i) {
        double* si = s + 3 * i;
        const double* hi = h + 3 * i;
        const double sh = si[0] * hi[0] + si[1] * hi[1] + si[2] * hi[2];
        double u[3];
        for (int c = 0; c < 3; ++c) u[c] = si[c] + dt * (hi[c] - sh * si[c]);
        const double n = sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
        for (int c = 0; c < 3; ++c) si[c] = u[c] / n;
    }
}

/* Eqs. 11-12 and the interpolation onto the uniform grid (Sec. III).
 *   s_0 = 0, s_k = s_{k-1} + ||phi*_k - phi*_{k-1}|| (Euclidean over all 3N components),
 *   alpha*_k = s_k / s_{K-1}, targets alpha_k = k/(K-1);
 *   for 0 < k < K-1: j = largest index with alpha*_j <= alpha_k, t = (alpha_k - alpha*_j) /
 *   (alpha*_{j+1} - alpha*_j), phi_k = per-site normalise((1-t) phi*_j + t phi*_{j+1});
 *   phi_0 and phi_{K-1} are kept; if s_{K-1} == 0 the path is returned unchanged.
 * phi_star and phi are [K][N][3] and must not overlap.  alpha_out (K entries, may be NULL)
 * receives alpha*. */
void or_reparam(int K, int n_sites, const double* phi_star, double* phi, double* alpha_out) {
    const size_t M = (size_t)3 * n_sites;
    double* sk = (double*)malloc(sizeof(double) * K);
    sk[0] = 0.0;
    for (int k = 1; k < K; ++k) {
        double d2 = 0.0;
        for (size_t c = 0; c < M; ++c) {
            const double d = phi_star[k * M + c] - phi_star[(k - 1) * M + c];
            d2 += d * d;
        }
        sk[k] = sk[k - 1] + sqrt(d2);
    }
    memcpy(phi, phi_star, sizeof(double) * M * K);
    if (sk[K - 1] == 0.0) {
        if (alpha_out)
            for (int k = 0; k < K; ++k) alpha_out[k] = 0.0;
        free(sk);
        return;
    }
    for (int k = 0; k < K; ++k) sk[k] = sk[k] / sk[K - 1];
    if (alpha_out) memcpy(alpha_out, sk, sizeof(double) * K);
    for (int k = 1; k < K - 1; ++k) {
        const double ak = (double)k / (double)(K - 1);
        int j = 0;
        for (int i = 0; i <= K - 2; ++i)
            if (sk[i] <= ak) j = i;
        const double t = (ak - sk[j]) / (sk[j + 1] - sk[j]);
        for (int i = 0; i < n_sites; ++i) {
            double u[3];
            for (int c = 0; c < 3; ++c) u[c] = (1.0 - t) * phi_star[j * M + 3 * i + c] + t * phi_star[(j + 1) * M + 3 * i + c];
            const double n = sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
            for (int c = 0; c < 3; ++c) phi[k * M + 3 * i + c] = u[c] / n;
        }
    }
    free(sk);
}

/* The string iteration of Sec. III: n_iter times { every image takes one step (Eq. 10/13) on its
 * own field (Eqs. 2-7); then the images are reparametrised to equal arc length (Eqs. 11-12) }.
 * `phi` ([K][N][3]) is updated in place.  When `energies` is not NULL it receives the energy
 * (Eq. 8) of every image of the final string, from a fresh field evaluation.
 * Returns 0, or -1 when out of memory. */
int or_string_run(const or_model* m, int K, int n_iter, double dt, double* phi, double* energies) {
    const int N = m->nx * m->ny * m->nz;
    const size_t M = (size_t)3 * N;
    double* table = NULL;
    if (m->w != 0.0) {
        table = dipole_table(m);
        if (!table) return -1;
    }
    double* h = (double*)malloc(sizeof(double) * M * K);
    double* star = (double*)malloc(sizeof(double) * M * K);
    if (!h || !star) {
        free(table);
        free(h);
        free(star);
        return -1;
    }
    for (int it = 0; it < n_iter; ++it) {
#pragma omp parallel for schedule(dynamic, 1)
        for (int k = 0; k < K; ++k) {
            field_one(m, table, phi + k * M, h + k * M);
            or_step(N, dt, h + k * M, phi + k * M);
        }
        memcpy(star, phi, sizeof(double) * M * K);
        or_reparam(K, N, star, phi, NULL);
    }
    if (energies) {
#pragma omp parallel for schedule(dynamic, 1)
        for (int k = 0; k < K; ++k) {
            field_one(m, table, phi + k * M, h + k * M);
            energies[k] = or_energy_from_field(N, phi + k * M, h + k * M);
        }
    }
    free(table);
    free(h);
    free(star);
    return 0;
}

/* ---- reparametrisation variants and the climbing image ------------------------------------------
 * Sec. III leaves the interpolation scheme open and names the climbing image as a refinement of the
 * saddle that the paper itself omits.  Readings taken here:
 *  - spline: a natural cubic spline (second derivative zero at both ends) through (alpha*_j, phi*_j),
 *    j over the part, per Cartesian component, evaluated at the targets and renormalised per site;
 *    a part with a zero-length segment, or with a single segment, is interpolated linearly;
 *  - climbing image kc (0 < kc < K-1): the string is reparametrised as two parts [0, kc] and
 *    [kc, K-1], each to equal arc length on its own (targets (k - a) / (b - a) in part [a, b]); kc
 *    itself does not move;
 *  - its dynamics: the projected force F = h - (s.h) s with its component along the unit tangent
 *    reversed, F - 2 (F.tau) tau / (tau.tau), tau = (phi_{kc+1} - phi_{kc-1}) projected per site onto
 *    the tangent plane at phi_kc, all from the states before the step; one Euler step of dt;
 *  - which image climbs: the interior image of highest energy among the states the previous
 *    iteration started from (lowest index on ties); none in the first iteration. */

/* Natural cubic spline second derivatives m[0..n] of (x_j, y_j), j = 0..n (n >= 2, x increasing):
 * m_0 = m_n = 0 and, for 0 < i < n, h_{i-1} m_{i-1} + 2 (h_{i-1} + h_i) m_i + h_i m_{i+1}
 * = 6 ((y_{i+1} - y_i) / h_i - (y_i - y_{i-1}) / h_{i-1}), h_i = x_{i+1} - x_i, solved by forward
 * elimination and back substitution (cp, dp: scratch of n + 1). */
static void natural_spline(int n, const double* x, const double* y, double* m, double* cp, double* dp) {
    m[0] = m[n] = 0.0;
    for (int i = 1; i < n; ++i) {
        const double hl = x[i] - x[i - 1], hr = x[i + 1] - x[i];
        const double diag = 2.0 * (hl + hr), rhs = 6.0 * ((y[i + 1] - y[i]) / hr - (y[i] - y[i - 1]) / hl);
        const double lo = i > 1 ? hl : 0.0;  /* coefficient of m_{i-1} (m_0 = 0 is known) */
        const double den = diag - lo * (i > 1 ? cp[i - 1] : 0.0);
        cp[i] = (i < n - 1 ? hr : 0.0) / den;
        dp[i] = (rhs - lo * (i > 1 ? dp[i - 1] : 0.0)) / den;
    }
    for (int i = n - 1; i >= 1; --i) m[i] = dp[i] - (i < n - 1 ? cp[i] * m[i + 1] : 0.0);
}

/* The spline of (x_j, y_j) with second derivatives m, on segment [x_j, x_{j+1}], at xe. */
static double spline_at(const double* x, const double* y, const double* m, int j, double xe) {
    const double h = x[j + 1] - x[j], a = x[j + 1] - xe, b = xe - x[j];
    return m[j] * a * a * a / (6.0 * h) + m[j + 1] * b * b * b / (6.0 * h) + (y[j] - m[j] * h * h / 6.0) * a / h +
           (y[j + 1] - m[j + 1] * h * h / 6.0) * b / h;
}

/* Reparametrisation (Eqs. 11-12) with the variants above: spline != 0 for the cubic spline, kc the
 * climbing image or -1.  alpha_out (optional, K): alpha*_k within its part. */
void or_reparam_v(int K, int n_sites, const double* phi_star, double* phi, int spline, int kc, double* alpha_out) {
    const size_t M = (size_t)3 * n_sites;
    double* sk = (double*)malloc(sizeof(double) * K * 6);
    double *al = sk + K, *y = sk + 2 * K, *mm = sk + 3 * K, *cp = sk + 4 * K, *dp = sk + 5 * K;
    sk[0] = 0.0;
    for (int k = 1; k < K; ++k) {
        double d2 = 0.0;
        for (size_t c = 0; c < M; ++c) {
            const double d = phi_star[k * M + c] - phi_star[(k - 1) * M + c];
            d2 += d * d;
        }
        sk[k] = sk[k - 1] + sqrt(d2);
    }
    memcpy(phi, phi_star, sizeof(double) * M * K);
    for (int k = 0; k < K; ++k) al[k] = 0.0;
    const int split = kc > 0 && kc < K - 1;
    const int parts[2][2] = {{0, split ? kc : K - 1}, {kc, K - 1}};
    for (int p = 0; p < 1 + split; ++p) {
        const int a = parts[p][0], b = parts[p][1], n = b - a;
        const double L = sk[b] - sk[a];
        if (!(L > 0.0)) continue;
        for (int j = a; j <= b; ++j) al[j] = (sk[j] - sk[a]) / L;
        int use_spline = spline && n >= 2;
        for (int j = a; j < b; ++j)
            if (!(al[j + 1] > al[j])) use_spline = 0;
        for (int k = a + 1; k < b; ++k) {
            const double ak = (double)(k - a) / (double)n;
            int j = a;
            for (int i = a; i <= b - 1; ++i)
                if (al[i] <= ak) j = i;
            const double t = (ak - al[j]) / (al[j + 1] - al[j]);
            for (int i = 0; i < n_sites; ++i) {
                double u[3];
                for (int c = 0; c < 3; ++c) {
                    if (use_spline) {
                        for (int q = 0; q <= n; ++q) y[q] = phi_star[(a + q) * M + 3 * i + c];
                        natural_spline(n, al + a, y, mm, cp, dp);
                        u[c] = spline_at(al + a, y, mm, j - a, ak);
                    } else {
                        u[c] = (1.0 - t) * phi_star[j * M + 3 * i + c] + t * phi_star[(j + 1) * M + 3 * i + c];
                    }
                }
                const double nr = sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
                for (int c = 0; c < 3; ++c) phi[k * M + 3 * i + c] = u[c] / nr;
            }
        }
    }
    if (alpha_out) memcpy(alpha_out, al, sizeof(double) * K);
    free(sk);
}

/* The string iteration of Sec. III with the variants above (Euler step as in or_string_run).  kc_out
 * (optional): the climbing image the next iteration would use, or -1. */
int or_string_run_v(const or_model* m, int K, int n_iter, double dt, int spline, int climb, double* phi,
                    double* energies, int* kc_out) {
    const int N = m->nx * m->ny * m->nz;
    const size_t M = (size_t)3 * N;
    double* table = NULL;
    if (m->w != 0.0) {
        table = dipole_table(m);
        if (!table) return -1;
    }
    double* h = (double*)malloc(sizeof(double) * M * K);
    double* star = (double*)malloc(sizeof(double) * M * K);
    double* sc = (double*)malloc(sizeof(double) * M);
    double* e = (double*)malloc(sizeof(double) * K);
    if (!h || !star || !sc || !e) {
        free(table);
        free(h);
        free(star);
        free(sc);
        free(e);
        return -1;
    }
    int kc = -1;
    for (int it = 0; it < n_iter; ++it) {
#pragma omp parallel for schedule(dynamic, 1)
        for (int k = 0; k < K; ++k) {
            field_one(m, table, phi + k * M, h + k * M);
            e[k] = or_energy_from_field(N, phi + k * M, h + k * M);
        }
        if (kc >= 0) {
            /* the climbing image's step, from the states before the step */
            const double *s = phi + kc * M, *hk = h + kc * M, *pp = phi + (kc + 1) * M, *pm = phi + (kc - 1) * M;
            double ft = 0.0, tt = 0.0;
            for (int i = 0; i < N; ++i) {
                const double* si = s + 3 * i;
                double tau[3], F[3];
                const double sh = si[0] * hk[3 * i] + si[1] * hk[3 * i + 1] + si[2] * hk[3 * i + 2];
                for (int c = 0; c < 3; ++c) {
                    tau[c] = pp[3 * i + c] - pm[3 * i + c];
                    F[c] = hk[3 * i + c] - sh * si[c];
                }
                const double ts = tau[0] * si[0] + tau[1] * si[1] + tau[2] * si[2];
                for (int c = 0; c < 3; ++c) {
                    tau[c] -= ts * si[c];
                    ft += F[c] * tau[c];
                    tt += tau[c] * tau[c];
                }
            }
            const double cf = tt > 0.0 ? ft / tt : 0.0;
            for (int i = 0; i < N; ++i) {
                const double* si = s + 3 * i;
                const double sh = si[0] * hk[3 * i] + si[1] * hk[3 * i + 1] + si[2] * hk[3 * i + 2];
                double tau[3], u[3];
                for (int c = 0; c < 3; ++c) tau[c] = pp[3 * i + c] - pm[3 * i + c];
                const double ts = tau[0] * si[0] + tau[1] * si[1] + tau[2] * si[2];
                for (int c = 0; c < 3; ++c) {
                    tau[c] -= ts * si[c];
                    u[c] = si[c] + dt * (hk[3 * i + c] - sh * si[c] - 2.0 * cf * tau[c]);
                }
                const double nr = sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
                for (int c = 0; c < 3; ++c) sc[3 * i + c] = u[c] / nr;
            }
        }
        for (int k = 0; k < K; ++k)
            if (k != kc) or_step(N, dt, h + k * M, phi + k * M);
        if (kc >= 0) memcpy(phi + kc * M, sc, sizeof(double) * M);
        memcpy(star, phi, sizeof(double) * M * K);
        or_reparam_v(K, N, star, phi, spline, kc, NULL);
        kc = -1;
        if (climb && K >= 3) {
            kc = 1;
            for (int k = 2; k < K - 1; ++k)
                if (e[k] > e[kc]) kc = k;
        }
    }
    if (kc_out) *kc_out = kc;
    if (energies) {
#pragma omp parallel for schedule(dynamic, 1)
        for (int k = 0; k < K; ++k) {
            field_one(m, table, phi + k * M, h + k * M);
            energies[k] = or_energy_from_field(N, phi + k * M, h + k * M);
        }
    }
    free(table);
    free(h);
    free(star);
    free(sc);
    free(e);
    return 0;
}

/* Adaptive explicit Runge-Kutta evolution of the images (Sec. III names explicit Runge-Kutta methods
 * with adaptive step-size control, namely the Dormand-Prince pair), in place of the fixed
 * projected-Euler step of or_string_run.  Each iteration integrates
 *     d phi_k / d tau = F(phi_k) = h(phi_k) - (phi_k . h(phi_k)) phi_k      (Eq. 13, every image k)
 * over the reduced interval T with the Dormand-Prince 5(4) pair, then reparametrises (Eqs. 11-12).
 * The images do not interact during the evolution, so the step control may treat them together or
 * apart: per_image = 0 integrates the whole string as one ODE system (one error norm, one step),
 * per_image = 1 gives every image its own system (its own norm and step).
 * Stage states are not renormalised (h is evaluated on them as they are); each accepted step is
 * followed by per-site renormalisation.  Error norm of a system: err = sqrt(mean_j (e_j / sc_j)^2)
 * over its components, e = step * sum_i (b_i - bhat_i) k_i, sc_j = atol + rtol * max(|y_j|, |y5_j|).
 * A step is accepted when err <= 1.  Next step: step * clamp(0.9 err^(-1/5), 0.2, 5) after an
 * accepted step, with the upper bound 1 after a rejected one; a non-finite err (stages that overflowed)
 * rejects with the factor 0.2.  Attempts are cut to end exactly at T.
 * step_io (one per system: 1, or K when per_image) carries the step from one iteration to the next
 * (set it to T before the first).  counts (optional, two per system): [accepted, rejected] summed over
 * the iterations.  Returns 0, -1 (memory), or -2 (more than 100000 attempts in one interval). */
static const double DP_A[7][6] = {
    {0, 0, 0, 0, 0, 0},
    {1.0 / 5.0, 0, 0, 0, 0, 0},
    {3.0 / 40.0, 9.0 / 40.0, 0, 0, 0, 0},
    {44.0 / 45.0, -56.0 / 15.0, 32.0 / 9.0, 0, 0, 0},
    {19372.0 / 6561.0, -25360.0 / 2187.0, 64448.0 / 6561.0, -212.0 / 729.0, 0, 0},
    {9017.0 / 3168.0, -355.0 / 33.0, 46732.0 / 5247.0, 49.0 / 176.0, -5103.0 / 18656.0, 0},
    {35.0 / 384.0, 0, 500.0 / 1113.0, 125.0 / 192.0, -2187.0 / 6784.0, 11.0 / 84.0}};
static const double DP_B[7] = {35.0 / 384.0, 0, 500.0 / 1113.0, 125.0 / 192.0, -2187.0 / 6784.0, 11.0 / 84.0, 0};
static const double DP_BHAT[7] = {5179.0 / 57600.0, 0,      7571.0 / 16695.0, 393.0 / 640.0, -92097.0 / 339200.0,
                                  187.0 / 2100.0,  1.0 / 40.0};

void or_dp_tableau(double a[7][6], double b[7], double bhat[7]) {
    memcpy(a, DP_A, sizeof(DP_A));
    memcpy(b, DP_B, sizeof(DP_B));
    memcpy(bhat, DP_BHAT, sizeof(DP_BHAT));
}

/* The Runge-Kutta-Fehlberg 4(5) pair (Fehlberg, 1969; Sec. III names it beside Dormand-Prince): six
 * stages, the fourth-order weights B4 (the solution carried forward, as in Fehlberg's method) and the
 * fifth-order weights B5 (the error estimate y5 - y4). */
static const double RKF_A[6][5] = {
    {0, 0, 0, 0, 0},
    {1.0 / 4.0, 0, 0, 0, 0},
    {3.0 / 32.0, 9.0 / 32.0, 0, 0, 0},
    {1932.0 / 2197.0, -7200.0 / 2197.0, 7296.0 / 2197.0, 0, 0},
    {439.0 / 216.0, -8.0, 3680.0 / 513.0, -845.0 / 4104.0, 0},
    {-8.0 / 27.0, 2.0, -3544.0 / 2565.0, 1859.0 / 4104.0, -11.0 / 40.0}};
static const double RKF_B4[6] = {25.0 / 216.0, 0, 1408.0 / 2565.0, 2197.0 / 4104.0, -1.0 / 5.0, 0};
static const double RKF_B5[6] = {16.0 / 135.0, 0, 6656.0 / 12825.0, 28561.0 / 56430.0, -9.0 / 50.0, 2.0 / 55.0};

void or_rkf_tableau(double a[6][5], double b4[6], double b5[6]) {
    memcpy(a, RKF_A, sizeof(RKF_A));
    memcpy(b4, RKF_B4, sizeof(RKF_B4));
    memcpy(b5, RKF_B5, sizeof(RKF_B5));
}

/* An embedded pair as the interval loop uses it: stage rows a (stage i uses a[i][0..i-1]), the weights
 * of the carried solution and the error weights (difference of the two solutions' weights). */
typedef struct {
    int stages;
    double a[7][6];
    double b[7];
    double e[7];
} rk_pair;

static rk_pair pair_of(int method) {
    rk_pair p;
    memset(&p, 0, sizeof p);
    if (method == 0) {
        p.stages = 7;
        memcpy(p.a, DP_A, sizeof(DP_A));
        for (int i = 0; i < 7; ++i) {
            p.b[i] = DP_B[i];
            p.e[i] = DP_B[i] - DP_BHAT[i];
        }
    } else {
        p.stages = 6;
        for (int i = 0; i < 6; ++i) {
            for (int j = 0; j < 5; ++j) p.a[i][j] = RKF_A[i][j];
            p.b[i] = RKF_B4[i];
            p.e[i] = RKF_B5[i] - RKF_B4[i];
        }
    }
    return p;
}

/* The right-hand side for every image of y (K images of M = 3N components) into f: F of Eq. 13 when
 * llg is NULL, else the reduced LLG of Eq. 9, f = -a (s x h) + b (h - (s.h) s) with a = llg[0] =
 * 1 / (1 + alpha^2) and b = llg[1] = alpha / (1 + alpha^2) (-s x (s x h) = h - (s.h) s). */
static void force_all(const or_model* m, const double* table, int K, const double* y, double* hbuf, double* f,
                      const double* llg) {
    const int N = m->nx * m->ny * m->nz;
    const size_t M = (size_t)3 * N;
#pragma omp parallel for schedule(dynamic, 1)
    for (int k = 0; k < K; ++k) {
        const double* yk = y + k * M;
        double* hk = hbuf + k * M;
        field_one(m, table, yk, hk);
        for (int i = 0; i < N; ++i) {
            const double* si = yk + 3 * i;
            const double* hi = hk + 3 * i;
            const double sh = si[0] * hi[0] + si[1] * hi[1] + si[2] * hi[2];
            double* fi = f + k * M + 3 * i;
            if (!llg) {
                for (int c = 0; c < 3; ++c) fi[c] = hi[c] - sh * si[c];
            } else {
                const double sxh[3] = {si[1] * hi[2] - si[2] * hi[1], si[2] * hi[0] - si[0] * hi[2],
                                       si[0] * hi[1] - si[1] * hi[0]};
                for (int c = 0; c < 3; ++c) fi[c] = -llg[0] * sxh[c] + llg[1] * (hi[c] - sh * si[c]);
            }
        }
    }
}

/* One interval [0, T] of the system of Ks images at phi (Ks * 3N components), DP 5(4) as above;
 * kk (7 systems), ys, y5 and hb are scratch of the system's size. */
static int rk_interval(const or_model* m, const double* table, const double* llg, const rk_pair* pr, int Ks,
                       double T, double rtol, double atol, double* step_io, double* phi, double* kk, double* ys,
                       double* y5, double* hb, long* acc, long* rej) {
    const int N = m->nx * m->ny * m->nz;
    const size_t M = (size_t)3 * N, L = M * (size_t)Ks;
    double step = *step_io, t = 0.0;
    int have_k1 = 0, attempts = 0;
    while (t < T) {
        if (++attempts > 100000) return -2;
        const double hs = step < T - t ? step : T - t;
        if (!have_k1) force_all(m, table, Ks, phi, hb, kk, llg);
        have_k1 = 1;
        for (int st = 1; st < pr->stages; ++st) {
            for (size_t j = 0; j < L; ++j) {
                double a = 0.0;
                for (int q = 0; q < st; ++q) a += pr->a[st][q] * kk[q * L + j];
                ys[j] = phi[j] + hs * a;
            }
            force_all(m, table, Ks, ys, hb, kk + st * L, llg);
        }
        double e2 = 0.0;
        for (size_t j = 0; j < L; ++j) {
            double b5 = 0.0, e = 0.0;
            for (int q = 0; q < pr->stages; ++q) {
                b5 += pr->b[q] * kk[q * L + j];
                e += pr->e[q] * kk[q * L + j];
            }
            y5[j] = phi[j] + hs * b5;
            const double ay = fabs(phi[j]), a5 = fabs(y5[j]);
            const double sc = atol + rtol * (ay > a5 ? ay : a5);
            const double r = hs * e / sc;
            e2 += r * r;
        }
        const double err = sqrt(e2 / (double)L);
        /* an attempt whose stages overflowed (the cubic growth of F off the unit sphere) is rejected
         * with the smallest factor */
        double fac = !isfinite(err) ? 0.2 : err > 0.0 ? 0.9 * pow(err, -0.2) : 5.0;
        if (fac < 0.2) fac = 0.2;
        if (err <= 1.0) {
            if (fac > 5.0) fac = 5.0;
            t = hs == T - t ? T : t + hs;
            for (size_t i = 0; i < L / 3; ++i) {
                const double* v = y5 + 3 * i;
                const double n = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
                for (int c = 0; c < 3; ++c) phi[3 * i + c] = v[c] / n;
            }
            have_k1 = 0;
            ++*acc;
        } else {
            if (fac > 1.0) fac = 1.0;
            ++*rej;
        }
        step = hs * fac;
    }
    *step_io = step;
    return 0;
}

/* The Runge-Kutta driver: n_iter intervals of T of the right-hand side chosen by llg (see force_all),
 * each followed by the reparametrisation when reparam != 0. */
static int run_rk(const or_model* m, int K, int n_iter, double T, double rtol, double atol, int method, int per_image,
                  const double* llg, int reparam, double* step_io, double* phi, double* energies, long* counts) {
    const rk_pair pr = pair_of(method);
    const int N = m->nx * m->ny * m->nz;
    const size_t M = (size_t)3 * N, L = M * (size_t)K;
    const int n_sys = per_image ? K : 1, Ks = per_image ? 1 : K;
    const size_t Ls = M * (size_t)Ks;
    double* table = NULL;
    if (m->w != 0.0) {
        table = dipole_table(m);
        if (!table) return -1;
    }
    double* kk = (double*)malloc(sizeof(double) * Ls * 7);
    double* ys = (double*)malloc(sizeof(double) * L);
    double* y5 = (double*)malloc(sizeof(double) * Ls);
    double* hb = (double*)malloc(sizeof(double) * L);
    long* cnt = (long*)calloc((size_t)2 * n_sys, sizeof(long));
    if (!kk || !ys || !y5 || !hb || !cnt) {
        free(table);
        free(kk);
        free(ys);
        free(y5);
        free(hb);
        free(cnt);
        return -1;
    }
    int rc = 0;
    for (int it = 0; it < n_iter && rc == 0; ++it) {
        for (int q = 0; q < n_sys && rc == 0; ++q)
            rc = rk_interval(m, table, llg, &pr, Ks, T, rtol, atol, step_io + q, phi + q * Ls, kk, ys, y5, hb,
                             &cnt[2 * q], &cnt[2 * q + 1]);
        if (rc) break;
        if (reparam) {
            memcpy(ys, phi, sizeof(double) * L);
            or_reparam(K, N, ys, phi, NULL);
        }
    }
    if (counts) memcpy(counts, cnt, sizeof(long) * 2 * n_sys);
    if (rc == 0 && energies) {
#pragma omp parallel for schedule(dynamic, 1)
        for (int k = 0; k < K; ++k) {
            field_one(m, table, phi + k * M, hb + k * M);
            energies[k] = or_energy_from_field(N, phi + k * M, hb + k * M);
        }
    }
    free(table);
    free(kk);
    free(ys);
    free(y5);
    free(hb);
    free(cnt);
    return rc;
}

int or_string_run_rk(const or_model* m, int K, int n_iter, double T, double rtol, double atol, int per_image,
                     double* step_io, double* phi, double* energies, long* counts) {
    return run_rk(m, K, n_iter, T, rtol, atol, 0, per_image, NULL, 1, step_io, phi, energies, counts);
}

/* As or_string_run_rk with the pair chosen by method: 0 Dormand-Prince 5(4), 1 Runge-Kutta-Fehlberg 4(5)
 * (the fourth-order solution carried forward). */
int or_string_run_rk_method(const or_model* m, int K, int n_iter, double T, double rtol, double atol, int method,
                            int per_image, double* step_io, double* phi, double* energies, long* counts) {
    return run_rk(m, K, n_iter, T, rtol, atol, method, per_image, NULL, 1, step_io, phi, energies, counts);
}

/* ---- precessional dynamics (Eq. 9) ------------------------------------------------------------------
 * In reduced units (h in units of J, time in units of mu0 |S| / (gamma J)) Eq. 9 reads
 *     ds/dtau = -1/(1 + alpha^2) s x h - alpha/(1 + alpha^2) s x (s x h),
 * every image an independent system and no reparametrisation.  or_llg_run: n_steps explicit Euler
 * steps s <- normalise(s + dt f(s)).  or_llg_run_rk: n_iter intervals of T with the Dormand-Prince pair
 * and the controller of or_string_run_rk.  energies (optional): Eq. 8 of the final states. */
int or_llg_run(const or_model* m, int K, int n_steps, double dt, double alpha, double* phi, double* energies) {
    const int N = m->nx * m->ny * m->nz;
    const size_t M = (size_t)3 * N, L = M * (size_t)K;
    const double llg[2] = {1.0 / (1.0 + alpha * alpha), alpha / (1.0 + alpha * alpha)};
    double* table = NULL;
    if (m->w != 0.0) {
        table = dipole_table(m);
        if (!table) return -1;
    }
    double* hb = (double*)malloc(sizeof(double) * L);
    double* f = (double*)malloc(sizeof(double) * L);
    if (!hb || !f) {
        free(table);
        free(hb);
        free(f);
        return -1;
    }
    for (int it = 0; it < n_steps; ++it) {
        force_all(m, table, K, phi, hb, f, llg);
        for (size_t i = 0; i < L / 3; ++i) {
            double u[3];
            for (int c = 0; c < 3; ++c) u[c] = phi[3 * i + c] + dt * f[3 * i + c];
            const double nr = sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
            for (int c = 0; c < 3; ++c) phi[3 * i + c] = u[c] / nr;
        }
    }
    if (energies) {
#pragma omp parallel for schedule(dynamic, 1)
        for (int k = 0; k < K; ++k) {
            field_one(m, table, phi + k * M, hb + k * M);
            energies[k] = or_energy_from_field(N, phi + k * M, hb + k * M);
        }
    }
    free(table);
    free(hb);
    free(f);
    return 0;
}

int or_llg_run_rk(const or_model* m, int K, int n_iter, double T, double alpha, double rtol, double atol,
                  int per_image, double* step_io, double* phi, double* energies, long* counts) {
    const double llg[2] = {1.0 / (1.0 + alpha * alpha), alpha / (1.0 + alpha * alpha)};
    return run_rk(m, K, n_iter, T, rtol, atol, 0, per_image, llg, 0, step_io, phi, energies, counts);
}

/* Sec. III: the barrier is the energy of the highest image relative to the first image.  Ties go
 * to the lowest index. */
double or_barrier(int K, const double* energies, int* k_max) {
    int kb = 0;
    for (int k = 1; k < K; ++k)
        if (energies[k] > energies[kb]) kb = k;
    if (k_max) *k_max = kb;
    return energies[kb] - energies[0];
}

/* Eq. 1 is linear in (J, D, K, w): out = (dE/dJ, dE/dD, dE/dK, dE/dw) of one image, each the
 * corresponding term of or_energy_terms evaluated with that constant set to 1. */
void or_energy_param_grad(const or_model* m, const double* s, double out[4]) {
    or_model u = *m;
    u.J = 1.0;
    u.D = 1.0;
    u.K = 1.0;
    u.w = 1.0;
    double t[5];
    or_energy_terms(&u, s, t);
    out[0] = t[0];
    out[1] = t[1];
    out[2] = t[2];
    out[3] = t[3];
}

/* Threads the OpenMP loops above may use (1 when built without OpenMP). */
int or_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void or_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}
