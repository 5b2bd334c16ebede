/*
 * FP64 oracle for the Monte Carlo Feynman-Kac evaluation of the TE
 * (E-polarisation) equation at interface nodes (Bihlo, Farquharson, Haynes,
 * Loredo-Osti, "Stochastic domain decomposition for the solution of the
 * two-dimensional magnetotelluric problem", arXiv:1603.09311).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow reference that the
 * CUDA path is checked against.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load it.  It shares no code, header,
 * table or constant generator with the CUDA library.
 *
 * Problem (Sec. 2.2, Eq. for the discontinuous elliptic problem and its TE
 * mapping): with the diffusion constant over the whole domain, TE reduces to
 *     (1/2) Lap u - (i kappa(x)/2) u = 0 in Omega,   u = g on dOmega,
 * whose Feynman-Kac solution (Kac-Feynman formula, Sec. 2.2) is
 *     u(x) = E[ g(beta_tau) exp(-i (1/2) int_0^tau kappa(beta_s) ds) ],
 * beta a standard 2D Brownian motion (generator Lap/2).  kappa here is the
 * dimensionless phase rate omega*mu*sigma*L^2 of each material.
 *
 * Discrete algorithm (Sec. 3.1), for node x0 and path r:
 *   1. beta = x0, n = 0, T_m = 0 (occupation step counts per material).
 *   2. Euler-Maruyama provisional step (Eq. for the discretised process):
 *        beta' = beta + sqrt(dt) * W,  W ~ N(0, I2)  (Box-Muller normals).
 *   3. Boundary reached by overshoot (beta' on or beyond a wall): the hit time
 *      is the linear-interpolation case of the first-hitting-time estimate
 *      (second case of the first-exit-time equation), theta_w = d/(d+|d'|).
 *   4. Both ends inside: Brownian-bridge test of the first case of the same
 *      equation with kappa_i = 1 applied to each wall of dOmega (Sec. 3.1,
 *      last paragraph before the Remark): t_w = -2 d d'/log U <= dt.
 *   5. Not exited: dt is added to the occupation time of the material in
 *      which beta' lies (Sec. 3.1, no regime change when the diffusion
 *      coefficients agree), beta = beta', n += 1.  (Pinned by one- and
 *      four-step walks beside a material edge: the count lands in the
 *      material with the Gaussian probability of the step's end point.)
 *   6. On exit at fraction theta of the step: the partial time theta*dt is
 *      charged to the material of beta^n, the exit point is the interpolated
 *      point beta + theta (beta' - beta) placed exactly on the hit wall, and
 *      the sample is g(exit) * exp(-i (1/2) sum_m kappa_m T_m) (the Monte
 *      Carlo estimator of Sec. 3.1).
 *
 * Random numbers: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), key =
 * the 64-bit seed, counter = (n>>1, r, node, 0) for the two words (a, b) of
 * step n (words 0,1 for even n, words 2,3 for odd n).  urule 32 (the
 * double-precision stream): normals from u = (w + 1/2) 2^-32 of a and b, the
 * bridge uniform from word 0 of counter (n, r, node, 1).  urule 23 (the
 * single-precision stream): normals from u = (w mod 2^23 + 1/2) 2^-23, the
 * bridge uniform from the remaining 18 bits, ((a>>23) 2^9 + (b>>23) + 1/2) 2^-18.
 * The paper fixes no random-number mapping; these are the library's.
 *
 * TM mode (diffusion coefficient that jumps; Sec. 2.2, Eq. for the Helmholtz
 * equation per sub-domain (1/2) kappa_i Lap u - lambda_i u = 0 with flux
 * continuity, and the interface rules of Sec. 3.1).  The sub-domains are
 * vertical strips (the paper treats one vertical interface "without loss of
 * generality"): strip m = [xif[m-1], xif[m]) has diffusion D_m and rates
 * kappa_{e,m}, i.e. D_m Lap u = i kappa_{e,m} u, and the walk weight keeps
 * the form exp(-i (1/2) sum_m kappa_{e,m} T_m).  Per step, in strip i:
 *   1. beta' = beta + sqrt(D_i dt) W (the discretised-process equation).
 *   2. dOmega first: overshoot as in TE; else the bridge with kappa_i = D_i
 *      for the wall of smallest w = 2 d d' / (D_i dt): hit iff U <= p_w,
 *      p_w = exp(-w) (0 when w > 40), U the step's bridge uniform.
 *   3. Interfaces to a strip of other D only (equal D: no regime change).
 *      Crossed: hitting fraction |d / (beta'_x - beta_x)| (second case of the
 *      first-hitting-time equation).  Not crossed: the bridge (first case)
 *      for the nearer such interface, g = 2 d d' / (D_i dt), with the
 *      uniform U_g = (U - p_w) / (1 - p_w) that the wall test leaves
 *      (uniform and independent of it given no wall hit): hit iff
 *      U <= p_w + (1 - p_w) p_g, p_g = exp(-g), and t_g = g dt / (-ln U_g).
 *      One uniform per step thus serves every barrier, as one serves all
 *      walls in TE.  A hit at fraction th resumes on side i with
 *      probability p_i = D_i / (D_i + D_j) (crossing-probability equation),
 *      uniformly in the disc of radius h = sqrt(dt max(D_i, D_j)) centred at
 *      (x_g -/+ h, z_g), z_g the hit height, tangent to the interface.
 *      Occupation: side i gets T_i += dt - (1/2)(dt - t_g) p_i,
 *      T_j += (1/2)(dt - t_g) p_i; side j gets T_i += t_g + (1/2)(dt - t_g) p_j
 *      and T_j the rest of dt (the printed T_j of that branch does not sum to
 *      dt with T_i; the reading keeps T_i and conserves dt).  A resampled
 *      point outside Omega ends the walk on the nearest wall (theta = 0).
 *   4. Otherwise dt goes to the strip of beta'.
 * A walk that starts on an interface between strips of different D has hit
 * it at time 0: its first step is the randomisation of 3 with t_g = 0, from
 * the strip on the left.
 * Pins (tests/test_oracle_pins.py): the flux-continuous solution int dx/D
 * (kappa = 0), the analytic test model, finite volumes with phase and flux,
 * equal D = the TE walk; the occupation split of step 3 by one-step walks
 * from a known distance of the interface (hit probability 2 Phi(-a/s) by the
 * reflection principle, mean occupation against its integral over the
 * Gaussian step and the hitting-time law) and from a start on it.
 * The TM uniforms U_alpha, disc radius and disc angle are words 1, 2, 3 of
 * the Philox call with counter (n, r, node, 2), by the urule.
 *
 * Build: gcc -O2 -std=c11 -ffp-contract=off -fopenmp -shared -fPIC.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_MAX_K 8
#define ORC_MAX_E 32

typedef struct {
    double xmin, xmax, zmin, zmax;   /* rectangular domain, z positive down */
    int K;                           /* number of materials */
    int E;                           /* number of evaluations (kappa rows) */
    const double *kappa;             /* [E][K] phase rates */
    int bg_air, bg_earth;            /* background material for z<0 / z>=0 */
    int n_shapes;
    const int *shape_kind;           /* 0 = rectangle [v0,v1)x[v2,v3), 1 = closed triangle */
    const int *shape_mat;
    const double *shape_v;           /* [n_shapes][6] */
    const int8_t *raster;            /* [nz][nx] material ids, or NULL */
    int nx, nz;
    int g_kind;                      /* 0 = 1D columns, 1 = complex affine, 2 = x^2 - z^2 */
    int g_left, g_right;             /* materials giving the column rates (g_kind 0) */
    const double *g_coef;            /* g_kind 1: a_re a_im b_re b_im c_re c_im */
    int urule;                       /* 32 or 23 */
    int64_t max_steps;
    int tm;                          /* 0 = TE; 1 = TM strips */
    const double *diff;              /* TM: [K] diffusion coefficient of strip m */
    const double *xif;               /* TM: [K-1] increasing strip boundaries */
} orc_model;

typedef struct {
    int64_t steps;       /* Euler steps taken, the exiting one included */
    double ex, ez;       /* exit point */
    double theta;        /* fraction of the last step before the hit */
    int wall;            /* 0 left, 1 right, 2 top, 3 bottom, -1 truncated */
    int m_last;          /* material of beta^n (gets theta*dt) */
    int truncated;
    int64_t count[ORC_MAX_K];
    double occ[ORC_MAX_K];   /* TM: occupation time per strip in units of dt */
    int64_t hits;            /* TM: interface randomisations */
} orc_walk_rec;

/* ---------------------------------------------------------------- Philox */

/* Philox4x32-10 as defined by Salmon et al. (SC'11): ten rounds of two
 * 32x32->64 multiplications by 0xD2511F53 and 0xCD9E8D57, with the key
 * bumped by the Weyl constants 0x9E3779B9 and 0xBB67AE85 between rounds. */
void orc_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

double orc_uniform(uint32_t w, int urule)
{
    if (urule == 23)
        return ((double)(w & 0x7fffffu) + 0.5) * (1.0 / 8388608.0);
    return ((double)w + 0.5) * (1.0 / 4294967296.0);
}

static void seed_key(uint64_t seed, uint32_t key[2])
{
    key[0] = (uint32_t)(seed & 0xffffffffu);
    key[1] = (uint32_t)(seed >> 32);
}

/* The two Philox words of step n of walk (node, path). */
static void step_words(uint64_t seed, uint32_t node, uint32_t path, int64_t n, uint32_t *a,
                       uint32_t *b)
{
    uint32_t key[2], ctr[4], x[4];
    seed_key(seed, key);
    ctr[0] = (uint32_t)(n >> 1); ctr[1] = path; ctr[2] = node; ctr[3] = 0;
    orc_philox4x32_10(ctr, key, x);
    *a = (n & 1) ? x[2] : x[0];
    *b = (n & 1) ? x[3] : x[1];
}

/* The two standard normals driving step n of walk (node, path). */
void orc_normals(uint64_t seed, uint32_t node, uint32_t path, int64_t n, int urule,
                 double *w0, double *w1)
{
    uint32_t a, b;
    step_words(seed, node, path, n, &a, &b);
    double u0 = orc_uniform(a, urule);
    double u1 = orc_uniform(b, urule);
    /* Box-Muller (1958): radius sqrt(-2 ln u0), angle 2 pi u1 */
    double rho = sqrt(-2.0 * log(u0));
    double ang = 6.283185307179586 * u1;
    *w0 = rho * cos(ang);
    *w1 = rho * sin(ang);
}

/* The uniform U_gamma of the Brownian-bridge test of step n.  urule 23: the
 * 18 bits of the step's two words that its normals leave unused,
 * U = ((a >> 23) * 2^9 + (b >> 23) + 1/2) 2^-18.  urule 32: word 0 of the
 * Philox call with counter (n, path, node, 1). */
double orc_bridge_uniform(uint64_t seed, uint32_t node, uint32_t path, int64_t n, int urule)
{
    if (urule == 23) {
        uint32_t a, b;
        step_words(seed, node, path, n, &a, &b);
        return ((double)(((a >> 23) << 9) | (b >> 23)) + 0.5) * (1.0 / 262144.0);
    }
    uint32_t key[2], ctr[4], x[4];
    seed_key(seed, key);
    ctr[0] = (uint32_t)n; ctr[1] = path; ctr[2] = node; ctr[3] = 1;
    orc_philox4x32_10(ctr, key, x);
    return orc_uniform(x[0], urule);
}

/* The four words of the TM Philox call of step n (counter (n, path, node, 2))
 * as uniforms; words 1, 2, 3 are U_alpha (side), disc radius, disc angle. */
void orc_tm_uniforms(uint64_t seed, uint32_t node, uint32_t path, int64_t n, int urule,
                     double U[4])
{
    uint32_t key[2], ctr[4], x[4];
    seed_key(seed, key);
    ctr[0] = (uint32_t)n; ctr[1] = path; ctr[2] = node; ctr[3] = 2;
    orc_philox4x32_10(ctr, key, x);
    for (int k = 0; k < 4; ++k) U[k] = orc_uniform(x[k], urule);
}

/* ------------------------------------------------------------- materials */

/* TM: the strip of abscissa x. */
int orc_strip(const orc_model *m, double x)
{
    int k = 0;
    while (k < m->K - 1 && x >= m->xif[k]) ++k;
    return k;
}

static int in_shape(int kind, const double *v, double x, double z)
{
    if (kind == 0)
        return (x >= v[0] && x < v[1] && z >= v[2] && z < v[3]);
    /* closed triangle: the point is on the inner side of (or on) all edges */
    double ax = v[0], az = v[1], bx = v[2], bz = v[3], cx = v[4], cz = v[5];
    double area = (bx - ax) * (cz - az) - (bz - az) * (cx - ax);
    double s = area >= 0.0 ? 1.0 : -1.0;
    double e0 = s * ((bx - ax) * (z - az) - (bz - az) * (x - ax));
    double e1 = s * ((cx - bx) * (z - bz) - (cz - bz) * (x - bx));
    double e2 = s * ((ax - cx) * (z - cz) - (az - cz) * (x - cx));
    return (e0 >= 0.0 && e1 >= 0.0 && e2 >= 0.0);
}

int orc_material(const orc_model *m, double x, double z)
{
    if (m->tm) return orc_strip(m, x);
    if (m->raster) {
        double fx = floor((x - m->xmin) * ((double)m->nx / (m->xmax - m->xmin)));
        double fz = floor((z - m->zmin) * ((double)m->nz / (m->zmax - m->zmin)));
        int64_t ix = (int64_t)fx, iz = (int64_t)fz;
        if (ix < 0) ix = 0;
        if (ix > m->nx - 1) ix = m->nx - 1;
        if (iz < 0) iz = 0;
        if (iz > m->nz - 1) iz = m->nz - 1;
        return (int)m->raster[iz * (int64_t)m->nx + ix];
    }
    int mat = (z >= 0.0) ? m->bg_earth : m->bg_air;
    for (int s = 0; s < m->n_shapes; ++s)
        if (in_shape(m->shape_kind[s], m->shape_v + 6 * s, x, z))
            mat = m->shape_mat[s];
    return mat;
}

/* ------------------------------------------------------ Dirichlet data g */

/* 1D layered TE solution of u'' = i kappa u for a column with earth rate
 * kappa below z = 0 and kappa = 0 (air) above: u = exp(-k z) for z >= 0 and
 * u = 1 - k z for z < 0, k = sqrt(i kappa) with Re k >= 0 (the boundary data
 * of Sec. 2.1: one-dimensional half-space solution on the sides). */
static double complex column_u(double kap, double z)
{
    double complex k = csqrt(I * kap);
    if (z >= 0.0)
        return cexp(-k * z);
    return 1.0 - k * z;
}

double complex orc_g_value(const orc_model *m, int e, int wall, double x, double z)
{
    if (m->g_kind == 1) {
        const double *c = m->g_coef;
        return (c[0] + I * c[1]) + (c[2] + I * c[3]) * x + (c[4] + I * c[5]) * z;
    }
    if (m->g_kind == 2)
        return x * x - z * z;
    if (m->g_kind == 3) {
        /* TM analytic test (Sec. 4.1, closed form read as (z + 1) cosh(a x)
         * with D a^2 = i kappa per strip): solves D Lap u = i kappa u in each
         * strip, continuous with zero flux at an interface at x = 0 */
        int st = orc_strip(m, x);
        double complex a = csqrt(I * m->kappa[e * m->K + st] / m->diff[st]);
        return (z + 1.0) * ccosh(a * x);
    }
    if (m->g_kind == 4) {
        /* TM, kappa = 0: u(x) = int_{xmin}^x ds / D(s), continuous with the
         * same flux D u' = 1 in every strip */
        double u = 0.0, a = m->xmin;
        for (int k = 0; k < m->K; ++k) {
            double b = (k < m->K - 1) ? m->xif[k] : m->xmax;
            if (x <= b) return u + (x - a) / m->diff[k];
            u += (b - a) / m->diff[k];
            a = b;
        }
        return u;
    }
    double kl = m->kappa[e * m->K + m->g_left];
    double kr = m->kappa[e * m->K + m->g_right];
    if (wall == 0)
        return column_u(kl, z);
    if (wall == 1)
        return column_u(kr, z);
    /* top and bottom: linear interpolation between the two corner values
     * (Sec. 2.1) */
    double t = (x - m->xmin) / (m->xmax - m->xmin);
    return (1.0 - t) * column_u(kl, z) + t * column_u(kr, z);
}

void orc_g(const orc_model *m, int e, int wall, double x, double z, double *re, double *im)
{
    double complex v = orc_g_value(m, e, wall, x, z);
    *re = creal(v);
    *im = cimag(v);
}

/* --------------------------------------------------------- the exit rule */

/* Distances of (x, z) to the walls left, right, top, bottom. */
static void wall_dist(const orc_model *m, double x, double z, double d[4])
{
    d[0] = x - m->xmin;
    d[1] = m->xmax - x;
    d[2] = z - m->zmin;
    d[3] = m->zmax - z;
}

static void place_on_wall(const orc_model *m, int wall, double x, double z, double xn,
                          double zn, double theta, double *ex, double *ez)
{
    *ex = x + theta * (xn - x);
    *ez = z + theta * (zn - z);
    if (wall == 0) *ex = m->xmin;
    if (wall == 1) *ex = m->xmax;
    if (wall == 2) *ez = m->zmin;
    if (wall == 3) *ez = m->zmax;
}

/* Exit test for the step beta=(x,z) -> beta'=(xn,zn) with bridge uniform U.
 * Returns 1 on exit and fills theta, wall and the exit point. */
int orc_exit_rule(const orc_model *m, double x, double z, double xn, double zn, double dt,
                  double U, double *theta, int *wall, double *ex, double *ez)
{
    double d[4], dn[4];
    wall_dist(m, x, z, d);
    wall_dist(m, xn, zn, dn);
    int over = 0;
    for (int w = 0; w < 4; ++w)
        if (dn[w] <= 0.0) over = 1;
    if (over) {
        /* linear interpolation of the hitting time, dt*|d/(beta'_perp - beta_perp)| */
        double best = INFINITY;
        int bw = -1;
        for (int w = 0; w < 4; ++w) {
            if (dn[w] <= 0.0) {
                double t = d[w] / (d[w] - dn[w]);
                if (t < best) { best = t; bw = w; }
            }
        }
        *theta = best;
        *wall = bw;
        place_on_wall(m, bw, x, z, xn, zn, best, ex, ez);
        return 1;
    }
    /* Brownian bridge: t_w = -2 d d' / log U <= dt  <=>  2 d d'/dt <= -log U */
    double best = INFINITY;
    int bw = -1;
    for (int w = 0; w < 4; ++w) {
        double e = 2.0 * d[w] * dn[w] / dt;
        if (e < best) { best = e; bw = w; }
    }
    double L = -log(U);
    if (best <= L) {
        *theta = best / L;
        *wall = bw;
        place_on_wall(m, bw, x, z, xn, zn, best / L, ex, ez);
        return 1;
    }
    return 0;
}

/* ------------------------------------------------------------- one walk */

void orc_walk(const orc_model *m, double x0, double z0, uint32_t node, uint32_t path,
              double dt, uint64_t seed, orc_walk_rec *rec)
{
    double sdt = sqrt(dt);
    double x = x0, z = z0;
    int64_t n = 0;
    memset(rec, 0, sizeof(*rec));
    for (;;) {
        if (n >= m->max_steps) {
            rec->steps = n;
            rec->truncated = 1;
            rec->wall = -1;
            rec->ex = x;
            rec->ez = z;
            rec->m_last = orc_material(m, x, z);
            return;
        }
        double w0, w1;
        orc_normals(seed, node, path, n, m->urule, &w0, &w1);
        double xn = x + sdt * w0;
        double zn = z + sdt * w1;
        double U = orc_bridge_uniform(seed, node, path, n, m->urule);
        double theta, ex, ez;
        int wall;
        if (orc_exit_rule(m, x, z, xn, zn, dt, U, &theta, &wall, &ex, &ez)) {
            rec->steps = n + 1;
            rec->ex = ex;
            rec->ez = ez;
            rec->theta = theta;
            rec->wall = wall;
            rec->m_last = orc_material(m, x, z);
            return;
        }
        rec->count[orc_material(m, xn, zn)] += 1;
        x = xn;
        z = zn;
        n += 1;
    }
}

/* One TM walk (the steps listed in the header). */
void orc_walk_tm(const orc_model *m, double x0, double z0, uint32_t node, uint32_t path,
                 double dt, uint64_t seed, orc_walk_rec *rec)
{
    double x = x0, z = z0;
    int i = orc_strip(m, x);
    int64_t n = 0;
    memset(rec, 0, sizeof(*rec));
    for (;;) {
        if (n >= m->max_steps) {
            rec->steps = n;
            rec->truncated = 1;
            rec->wall = -1;
            rec->ex = x;
            rec->ez = z;
            rec->m_last = i;
            return;
        }
        double w0, w1;
        orc_normals(seed, node, path, n, m->urule, &w0, &w1);
        double Di = m->diff[i];
        double s = sqrt(Di * dt);
        double xn = x + s * w0;
        double zn = z + s * w1;
        double U = orc_bridge_uniform(seed, node, path, n, m->urule);
        double ex, ez;
        double th = 2.0, xg = 0.0;
        int side = -1;
        double V[4];
        orc_tm_uniforms(seed, node, path, n, m->urule, V);
        int j = i;
        if (n == 0 && i > 0 && x == m->xif[i - 1] && m->diff[i - 1] != Di) {
            /* started on an interface: a hit at t_g = 0 from the left strip */
            i = i - 1;
            Di = m->diff[i];
            xn = x;
            zn = z;
            th = 0.0;
            side = i + 1;
            xg = x;
        } else {
            /* 2. the outer boundary first, with the strip's diffusion */
            double d[4], dn[4];
            wall_dist(m, x, z, d);
            wall_dist(m, xn, zn, dn);
            int over = 0;
            for (int w = 0; w < 4; ++w)
                if (dn[w] <= 0.0) over = 1;
            if (over) {
                double best = INFINITY;
                int bw = -1;
                for (int w = 0; w < 4; ++w)
                    if (dn[w] <= 0.0) {
                        double t = d[w] / (d[w] - dn[w]);
                        if (t < best) { best = t; bw = w; }
                    }
                rec->steps = n + 1;
                place_on_wall(m, bw, x, z, xn, zn, best, &rec->ex, &rec->ez);
                rec->theta = best;
                rec->wall = bw;
                rec->m_last = i;
                return;
            }
            double wmin = INFINITY;
            int bw = -1;
            for (int w = 0; w < 4; ++w) {
                double q = 2.0 * d[w] * dn[w] / (Di * dt);
                if (q < wmin) { wmin = q; bw = w; }
            }
            double pw = wmin <= 40.0 ? exp(-wmin) : 0.0;
            if (U <= pw) {
                double th_w = wmin / -log(U);
                rec->steps = n + 1;
                place_on_wall(m, bw, x, z, xn, zn, th_w, &rec->ex, &rec->ez);
                rec->theta = th_w;
                rec->wall = bw;
                rec->m_last = i;
                return;
            }
            /* 3. the interfaces of strip i */
            j = orc_strip(m, xn);
            if (j != i) {
                int jn = (j > i) ? i + 1 : i - 1;
                double xi = (j > i) ? m->xif[i] : m->xif[i - 1];
                if (m->diff[jn] != Di) {
                    th = fabs((x - xi) / (xn - x));
                    side = jn;
                    xg = xi;
                }
            } else {
                double g = INFINITY, bx = 0.0;
                int bs = -1;
                if (i > 0 && m->diff[i - 1] != Di) {
                    double e = 2.0 * (x - m->xif[i - 1]) * (xn - m->xif[i - 1]) / (Di * dt);
                    if (e < g) { g = e; bs = i - 1; bx = m->xif[i - 1]; }
                }
                if (i < m->K - 1 && m->diff[i + 1] != Di) {
                    double e = 2.0 * (m->xif[i] - x) * (m->xif[i] - xn) / (Di * dt);
                    if (e < g) { g = e; bs = i + 1; bx = m->xif[i]; }
                }
                double pg = (bs >= 0 && g <= 40.0) ? exp(-g) : 0.0;
                if (pg > 0.0 && U <= pw + (1.0 - pw) * pg) {
                    double Ug = (U - pw) / (1.0 - pw);
                    th = g / -log(Ug);
                    side = bs;
                    xg = bx;
                }
            }
        }
        if (side >= 0) {
            /* randomise the side (crossing probability), resample in the disc,
             * split the step's time */
            double Dj = m->diff[side];
            double pi_ = Di / (Di + Dj), pj = Dj / (Di + Dj);
            double zg = z + th * (zn - z);
            double h = sqrt(dt * (Di > Dj ? Di : Dj));
            double c = (x <= xg) ? h : -h;
            double rest = 1.0 - th, cx;
            if (V[1] < pi_) {
                rec->occ[i] += 1.0 - 0.5 * rest * pi_;
                rec->occ[side] += 0.5 * rest * pi_;
                cx = xg - c;
            } else {
                double ti = th + 0.5 * rest * pj;
                rec->occ[i] += ti;
                rec->occ[side] += 1.0 - ti;
                cx = xg + c;
            }
            double rho = h * sqrt(V[2]);
            double ang = 6.283185307179586 * V[3];
            xn = cx + rho * cos(ang);
            zn = zg + rho * sin(ang);
            rec->hits += 1;
            double dn[4];
            wall_dist(m, xn, zn, dn);
            int bw = -1;
            double most = 0.0;
            for (int w = 0; w < 4; ++w)
                if (dn[w] <= most && (bw < 0 || dn[w] < most)) { most = dn[w]; bw = w; }
            if (bw >= 0) {
                /* the resampled point left Omega: end on the nearest wall */
                ex = xn < m->xmin ? m->xmin : (xn > m->xmax ? m->xmax : xn);
                ez = zn < m->zmin ? m->zmin : (zn > m->zmax ? m->zmax : zn);
                if (bw == 0) ex = m->xmin;
                if (bw == 1) ex = m->xmax;
                if (bw == 2) ez = m->zmin;
                if (bw == 3) ez = m->zmax;
                rec->steps = n + 1;
                rec->ex = ex;
                rec->ez = ez;
                rec->theta = 0.0;
                rec->wall = bw;
                rec->m_last = i;
                return;
            }
            x = xn;
            z = zn;
            i = orc_strip(m, x);
            n += 1;
            continue;
        }
        /* 4. the step's time goes to the strip of beta' */
        rec->count[j] += 1;
        rec->occ[j] += 1.0;
        x = xn;
        z = zn;
        i = j;
        n += 1;
    }
}

/* Sample of one finished walk for evaluation e (Monte Carlo estimator of
 * Sec. 3.1): g(exit) * exp(-i (1/2) sum_m kappa_{e,m} T_m). */
double complex orc_sample(const orc_model *m, int e, const orc_walk_rec *rec, double dt)
{
    double phase = 0.0;
    for (int k = 0; k < m->K; ++k)
        phase += m->kappa[e * m->K + k] * ((m->tm ? rec->occ[k] : (double)rec->count[k]) * dt);
    phase += m->kappa[e * m->K + rec->m_last] * (rec->theta * dt);
    phase *= 0.5;
    double complex wgt = cexp(-I * phase);
    return wgt * orc_g_value(m, e, rec->wall, rec->ex, rec->ez);
}

/* ------------------------------------------------- interface-node values */

#define ORC_BLOCK 4096

typedef struct {
    double s_re[ORC_MAX_E], s_im[ORC_MAX_E], q_re[ORC_MAX_E], q_im[ORC_MAX_E];
    double s_tau;
    int64_t steps, walks, truncated;
} orc_partial;

/*
 * Monte Carlo values at n_nodes nodes.  Node j uses RNG node id
 * node_id0 + j and paths 0..n_paths[j]-1.  Outputs:
 *   mean[j][e][2]  (re, im) of the sample mean over non-truncated paths,
 *   se[j][e][2]    standard error of each component (unbiased variance / N),
 *   tau_mean[j]    mean of the estimated exit time (n + theta) dt (nullable),
 *   stats[3]       total steps, walks, truncated walks (nullable).
 * Paths are summed in blocks of ORC_BLOCK in fixed order, so the result does
 * not depend on the number of threads.  Returns the number of truncated walks.
 */
int64_t orc_interface_values(const orc_model *m, const double *nodes_xz, int n_nodes,
                             const int64_t *n_paths, uint32_t node_id0, double dt,
                             uint64_t seed, int n_threads, double *mean, double *se,
                             double *tau_mean, int64_t *stats)
{
    int64_t *blk0 = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n_nodes + 1));
    blk0[0] = 0;
    for (int j = 0; j < n_nodes; ++j)
        blk0[j + 1] = blk0[j] + (n_paths[j] + ORC_BLOCK - 1) / ORC_BLOCK;
    int64_t nblk = blk0[n_nodes];
    orc_partial *part = (orc_partial *)calloc((size_t)(nblk > 0 ? nblk : 1), sizeof(orc_partial));
#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
#endif
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t b = 0; b < nblk; ++b) {
        int j = 0;
        while (blk0[j + 1] <= b) ++j;
        int64_t p0 = (b - blk0[j]) * ORC_BLOCK;
        int64_t p1 = p0 + ORC_BLOCK;
        if (p1 > n_paths[j]) p1 = n_paths[j];
        orc_partial *P = &part[b];
        for (int64_t p = p0; p < p1; ++p) {
            orc_walk_rec rec;
            (m->tm ? orc_walk_tm : orc_walk)(m, nodes_xz[2 * j], nodes_xz[2 * j + 1],
                                             node_id0 + (uint32_t)j, (uint32_t)p, dt, seed, &rec);
            P->steps += rec.steps;
            P->walks += 1;
            if (rec.truncated) {
                P->truncated += 1;
                continue;
            }
            P->s_tau += ((double)(rec.steps - 1) + rec.theta) * dt;
            for (int e = 0; e < m->E; ++e) {
                double complex v = orc_sample(m, e, &rec, dt);
                double re = creal(v), im = cimag(v);
                P->s_re[e] += re;
                P->s_im[e] += im;
                P->q_re[e] += re * re;
                P->q_im[e] += im * im;
            }
        }
    }
    int64_t tot_steps = 0, tot_walks = 0, tot_trunc = 0;
    for (int j = 0; j < n_nodes; ++j) {
        orc_partial acc;
        memset(&acc, 0, sizeof(acc));
        for (int64_t b = blk0[j]; b < blk0[j + 1]; ++b) {
            for (int e = 0; e < m->E; ++e) {
                acc.s_re[e] += part[b].s_re[e];
                acc.s_im[e] += part[b].s_im[e];
                acc.q_re[e] += part[b].q_re[e];
                acc.q_im[e] += part[b].q_im[e];
            }
            acc.s_tau += part[b].s_tau;
            acc.steps += part[b].steps;
            acc.walks += part[b].walks;
            acc.truncated += part[b].truncated;
        }
        double N = (double)(acc.walks - acc.truncated);
        for (int e = 0; e < m->E; ++e) {
            double mr = N > 0 ? acc.s_re[e] / N : NAN;
            double mi = N > 0 ? acc.s_im[e] / N : NAN;
            mean[(j * m->E + e) * 2 + 0] = mr;
            mean[(j * m->E + e) * 2 + 1] = mi;
            double vr = NAN, vi = NAN;
            if (N > 1) {
                vr = (acc.q_re[e] - acc.s_re[e] * mr) / (N - 1.0);
                vi = (acc.q_im[e] - acc.s_im[e] * mi) / (N - 1.0);
                if (vr < 0) vr = 0;
                if (vi < 0) vi = 0;
            }
            se[(j * m->E + e) * 2 + 0] = sqrt(vr / N);
            se[(j * m->E + e) * 2 + 1] = sqrt(vi / N);
        }
        if (tau_mean) tau_mean[j] = N > 0 ? acc.s_tau / N : NAN;
        tot_steps += acc.steps;
        tot_walks += acc.walks;
        tot_trunc += acc.truncated;
    }
    if (stats) {
        stats[0] = tot_steps;
        stats[1] = tot_walks;
        stats[2] = tot_trunc;
    }
    free(part);
    free(blk0);
    return tot_trunc;
}

/* Raw sums of path ranges: range i is paths [path_begin[i], path_begin[i] +
 * path_count[i]) of the node at nodes_xz[i] with node id node_ids[i].  Per
 * range and evaluation: sum re, sum im, sum re^2, sum im^2 over the walks that
 * reached the boundary, added in path order (one range per thread, so the
 * sums do not depend on the number of threads); n_valid[i] those walks, and
 * stats[0] the Euler steps of all walks.  A range is the unit a sharded
 * evaluation hands to one process: every range's walks are independent of
 * the others (Sec. 5). */
void orc_range_sums(const orc_model *m, const double *nodes_xz, const uint32_t *node_ids,
                    int n_ranges, const int64_t *path_begin, const int64_t *path_count, double dt,
                    uint64_t seed, int n_threads, double *sums /* [n][E][4] */,
                    int64_t *n_valid, int64_t *stats)
{
    int64_t steps = 0;
#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
#endif
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : steps)
    for (int i = 0; i < n_ranges; ++i) {
        double *S = sums + (size_t)i * m->E * 4;
        for (int k = 0; k < m->E * 4; ++k) S[k] = 0.0;
        int64_t nv = 0;
        for (int64_t p = path_begin[i]; p < path_begin[i] + path_count[i]; ++p) {
            orc_walk_rec rec;
            (m->tm ? orc_walk_tm : orc_walk)(m, nodes_xz[2 * i], nodes_xz[2 * i + 1], node_ids[i],
                                             (uint32_t)p, dt, seed, &rec);
            steps += rec.steps;
            if (rec.truncated) continue;
            nv += 1;
            for (int e = 0; e < m->E; ++e) {
                double complex v = orc_sample(m, e, &rec, dt);
                double re = creal(v), im = cimag(v);
                S[4 * e + 0] += re;
                S[4 * e + 1] += im;
                S[4 * e + 2] += re * re;
                S[4 * e + 3] += im * im;
            }
        }
        n_valid[i] = nv;
    }
    if (stats) stats[0] = steps;
}

/* Per-path records of paths [p0, p0+count) of one node (for per-path
 * comparison of exit steps, counts and exit points). */
void orc_walk_records(const orc_model *m, double x0, double z0, uint32_t node, uint32_t p0,
                      int count, double dt, uint64_t seed, int n_threads, int64_t *steps,
                      int64_t *counts /* [count][K] */, double *exit_xzt /* [count][3] */,
                      int *wall, int *m_last, int *truncated, double *occ /* [count][K] */,
                      int64_t *hits)
{
#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
#endif
#pragma omp parallel for schedule(dynamic, 64)
    for (int i = 0; i < count; ++i) {
        orc_walk_rec rec;
        (m->tm ? orc_walk_tm : orc_walk)(m, x0, z0, node, p0 + (uint32_t)i, dt, seed, &rec);
        steps[i] = rec.steps;
        for (int k = 0; k < m->K; ++k)
            occ[(int64_t)i * m->K + k] = m->tm ? rec.occ[k] : (double)rec.count[k];
        hits[i] = rec.hits;
        for (int k = 0; k < m->K; ++k) counts[(int64_t)i * m->K + k] = rec.count[k];
        exit_xzt[3 * i + 0] = rec.ex;
        exit_xzt[3 * i + 1] = rec.ez;
        exit_xzt[3 * i + 2] = rec.theta;
        wall[i] = rec.wall;
        m_last[i] = rec.m_last;
        truncated[i] = rec.truncated;
    }
}

int orc_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
