/*
 * lb_oracle.c -- plain, slow FP64 CPU oracle for one time step of the
 * two-component D3Q19 BGK lattice-Boltzmann method with a Shan-Chen
 * inter-component force, streaming, periodic wrap and halfway bounce-back.
 *
 * TEST INFRASTRUCTURE. Only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark load this library. The CUDA product path
 * shares no code with it and never calls it.
 *
 * What each part follows:
 *   - D3Q19 velocity set: 19 velocities, rest + 6 at distance 1 + 12 at
 *     distance sqrt(2); the 8 corner velocities are dropped (Sec. 2, Method).
 *   - Weights w = 1/3, 1/18, 1/36 for |c|^2 = 0, 1, 2 and c_s^2 = 1/3
 *     (Appendix, table of D3Q19 coefficients; Eq. LEQ).
 *   - Per-component density rho^k = sum_i f_i^k and mixture momentum
 *     rho u = sum_k sum_i f_i^k c_i (Appendix, moments below Eq. CGLBE).
 *   - BGK relaxation f* = f - (f - f^eq)/tau with omega = 1/tau (Eq. bgk).
 *   - Second-order equilibrium (Eq. LEQ).
 *   - Streaming f_i(x + c_i) <- f*_i(x) (Eq. bgk, left-hand side).
 *   - Halfway bounce-back for a wall at rest: a population that would stream
 *     into a solid node comes back to its own node reversed (Eq. LADDFLBE
 *     with u_b = 0). Interior solid nodes hold no fluid (Sec. 2, Method).
 *   - Shan-Chen force with psi = rho: the paper gives none (its two-component
 *     model is the colour-gradient one); the standard pseudopotential form of
 *     Krueger et al. (2017), the LBM text the paper cites, is used:
 *         F^A(x) = -G psi^A(x) sum_{i=1..18} w_i psi^B(x + c_i) c_i
 *     and F^B with A and B swapped; psi = rho at fluid nodes and psi = 0 at
 *     solid nodes; optional body force F^k += rho^k g.
 *   - Forcing by the original Shan-Chen velocity shift: the common velocity
 *     u' = (sum_k sum_i c_i f_i^k / tau) / (sum_k rho^k / tau) and
 *     u_eq^k = u' + tau F^k / rho^k enter f^eq of component k.
 *
 * Step order (state = post-streaming, pre-collision populations f):
 *   C1 densities, C2 force, C3 velocities, C4 collision, C5 stream.
 *
 * Layout: f[(k*19 + i)*N + s], k in {0 = A, 1 = B}, s = x + nx*(y + ny*z).
 * Velocity order (the library's public order): 0 rest; 1..6 = +x,-x,+y,-y,
 * +z,-z; 7..18 the 12 diagonals in opposite pairs (7,8), (9,10), ..., (17,18).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define Q 19

/* the oracle's own copy of the velocity set */
static const int CV[Q][3] = {
    { 0, 0, 0},
    { 1, 0, 0}, {-1, 0, 0}, { 0, 1, 0}, { 0,-1, 0}, { 0, 0, 1}, { 0, 0,-1},
    { 1, 1, 0}, {-1,-1, 0}, { 1,-1, 0}, {-1, 1, 0},
    { 1, 0, 1}, {-1, 0,-1}, { 1, 0,-1}, {-1, 0, 1},
    { 0, 1, 1}, { 0,-1,-1}, { 0, 1,-1}, { 0,-1, 1},
};

static double W[Q];
static int OPP[Q];
static int lattice_ready = 0;

/* Weights from the coefficient table by |c|^2; the opposite direction by
 * search, so that neither is a hand-typed table. */
static void lattice_setup(void)
{
    if (lattice_ready) return;
    for (int i = 0; i < Q; ++i) {
        int c2 = CV[i][0]*CV[i][0] + CV[i][1]*CV[i][1] + CV[i][2]*CV[i][2];
        W[i] = (c2 == 0) ? 1.0/3.0 : (c2 == 1) ? 1.0/18.0 : 1.0/36.0;
        OPP[i] = -1;
        for (int j = 0; j < Q; ++j)
            if (CV[j][0] == -CV[i][0] && CV[j][1] == -CV[i][1] && CV[j][2] == -CV[i][2])
                OPP[i] = j;
    }
    lattice_ready = 1;
}

static inline int wrap(int a, int n) { a %= n; return a < 0 ? a + n : a; }

static inline long site(int x, int y, int z, int nx, int ny) {
    return (long)x + (long)nx * ((long)y + (long)ny * (long)z);
}

/* neighbour of (x,y,z) along +c_i with periodic wrap */
static inline long nbr(int x, int y, int z, int i, int nx, int ny, int nz) {
    return site(wrap(x + CV[i][0], nx), wrap(y + CV[i][1], ny), wrap(z + CV[i][2], nz), nx, ny);
}

static inline int is_fluid(const uint8_t* mask, long s) { return mask == NULL || mask[s] == 0; }

/* Eq. LEQ: w_i rho [1 + c.u/cs2 + (c.u)^2/(2 cs4) - u.u/(2 cs2)], cs2 = 1/3 */
static inline double feq(int i, double rho, const double u[3]) {
    const double cs2 = 1.0 / 3.0;
    double cu = CV[i][0]*u[0] + CV[i][1]*u[1] + CV[i][2]*u[2];
    double uu = u[0]*u[0] + u[1]*u[1] + u[2]*u[2];
    return W[i] * rho * (1.0 + cu/cs2 + cu*cu/(2.0*cs2*cs2) - uu/(2.0*cs2));
}

void oracle_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int oracle_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* The oracle's lattice, for the tests that pin it (isotropy sums). */
void oracle_lattice(int* c /* 57 */, double* w /* 19 */, int* opp /* 19 */) {
    lattice_setup();
    for (int i = 0; i < Q; ++i) {
        c[3*i] = CV[i][0]; c[3*i+1] = CV[i][1]; c[3*i+2] = CV[i][2];
        w[i] = W[i]; opp[i] = OPP[i];
    }
}

/* Initial populations: f_i^k = f_i^eq(rho^k, u) at fluid nodes, 0 at solid.
 * u may be NULL (zero velocity); otherwise SoA, u[a*N + s]. */
void oracle_init(int nx, int ny, int nz, const uint8_t* mask,
                 const double* rhoA, const double* rhoB, const double* u, double* f)
{
    lattice_setup();
    const long N = (long)nx * ny * nz;
    #pragma omp parallel for schedule(static)
    for (long s = 0; s < N; ++s) {
        double uu[3] = {0, 0, 0};
        if (u) { uu[0] = u[s]; uu[1] = u[N + s]; uu[2] = u[2*N + s]; }
        int fl = is_fluid(mask, s);
        for (int i = 0; i < Q; ++i) {
            f[(0*Q + i)*N + s] = fl ? feq(i, rhoA[s], uu) : 0.0;
            f[(1*Q + i)*N + s] = fl ? feq(i, rhoB[s], uu) : 0.0;
        }
    }
}

/* C1 + C2: densities rho[k*N + s] and Shan-Chen force F[(k*3 + a)*N + s]
 * (plus rho^k g when g != NULL). */
void oracle_density_force(int nx, int ny, int nz, double G, const double* g,
                          const uint8_t* mask, const double* f, double* rho, double* F)
{
    lattice_setup();
    const long N = (long)nx * ny * nz;
    /* C1 */
    #pragma omp parallel for schedule(static)
    for (long s = 0; s < N; ++s) {
        for (int k = 0; k < 2; ++k) {
            double r = 0.0;
            if (is_fluid(mask, s))
                for (int i = 0; i < Q; ++i) r += f[(k*Q + i)*N + s];
            rho[k*N + s] = r;   /* psi = rho at fluid nodes, 0 at solid nodes */
        }
    }
    /* C2 */
    #pragma omp parallel for schedule(static)
    for (int z = 0; z < nz; ++z)
    for (int y = 0; y < ny; ++y)
    for (int x = 0; x < nx; ++x) {
        long s = site(x, y, z, nx, ny);
        for (int k = 0; k < 2; ++k) {
            int kb = 1 - k;
            double sum[3] = {0, 0, 0};
            for (int i = 1; i < Q; ++i) {
                double psi_nb = rho[kb*N + nbr(x, y, z, i, nx, ny, nz)];
                for (int a = 0; a < 3; ++a) sum[a] += W[i] * psi_nb * CV[i][a];
            }
            for (int a = 0; a < 3; ++a) {
                double Fa = -G * rho[k*N + s] * sum[a];
                if (g && is_fluid(mask, s)) Fa += rho[k*N + s] * g[a];
                F[(k*3 + a)*N + s] = is_fluid(mask, s) ? Fa : 0.0;
            }
        }
    }
}

/* One full step f_in -> f_out (C1..C5). Returns 0, or 1 when a fluid node
 * has rho^k <= 0 (the force shift divides by rho^k). f_in and f_out must not
 * alias. */
int oracle_step(int nx, int ny, int nz, double tau, double G, const double* g,
                const uint8_t* mask, const double* f_in, double* f_out)
{
    lattice_setup();
    const long N = (long)nx * ny * nz;
    double* rho = (double*)malloc(sizeof(double) * 2 * N);
    double* F = (double*)malloc(sizeof(double) * 6 * N);
    double* fpost = (double*)malloc(sizeof(double) * 2 * Q * N);
    if (!rho || !F || !fpost) { free(rho); free(F); free(fpost); return 2; }
    int bad = 0;

    oracle_density_force(nx, ny, nz, G, g, mask, f_in, rho, F);

    /* C3 + C4 */
    #pragma omp parallel for schedule(static) reduction(|:bad)
    for (long s = 0; s < N; ++s) {
        if (!is_fluid(mask, s)) {
            for (int j = 0; j < 2*Q; ++j) fpost[j*N + s] = 0.0;
            continue;
        }
        double rA = rho[s], rB = rho[N + s];
        if (!(rA > 0.0) || !(rB > 0.0)) { bad = 1; continue; }
        double mom[3] = {0, 0, 0};
        for (int k = 0; k < 2; ++k)
            for (int i = 0; i < Q; ++i)
                for (int a = 0; a < 3; ++a) mom[a] += CV[i][a] * f_in[(k*Q + i)*N + s];
        /* u' = (sum_k j^k / tau) / (sum_k rho^k / tau) */
        double up[3];
        for (int a = 0; a < 3; ++a) up[a] = (mom[a] / tau) / (rA / tau + rB / tau);
        for (int k = 0; k < 2; ++k) {
            double rk = rho[k*N + s];
            double ueq[3];
            for (int a = 0; a < 3; ++a) ueq[a] = up[a] + tau * F[(k*3 + a)*N + s] / rk;
            for (int i = 0; i < Q; ++i) {
                double fi = f_in[(k*Q + i)*N + s];
                fpost[(k*Q + i)*N + s] = fi - (fi - feq(i, rk, ueq)) / tau;
            }
        }
    }

    /* C5: push each post-collision population along c_i; a population that
     * would land on a solid node is reflected into the opposite direction
     * at its own node. */
    memset(f_out, 0, sizeof(double) * 2 * Q * N);
    #pragma omp parallel for schedule(static)
    for (int z = 0; z < nz; ++z)
    for (int y = 0; y < ny; ++y)
    for (int x = 0; x < nx; ++x) {
        long s = site(x, y, z, nx, ny);
        if (!is_fluid(mask, s)) continue;
        for (int k = 0; k < 2; ++k)
            for (int i = 0; i < Q; ++i) {
                long d = nbr(x, y, z, i, nx, ny, nz);
                double v = fpost[(k*Q + i)*N + s];
                if (is_fluid(mask, d)) f_out[(k*Q + i)*N + d] = v;
                else                   f_out[(k*Q + OPP[i])*N + s] = v;
            }
    }
    free(rho); free(F); free(fpost);
    return bad;
}

/* n steps in place on f (ping-pong through an internal buffer). */
int oracle_run(int nx, int ny, int nz, double tau, double G, const double* g,
               const uint8_t* mask, int nsteps, double* f)
{
    const long N = (long)nx * ny * nz;
    double* tmp = (double*)malloc(sizeof(double) * 2 * Q * N);
    if (!tmp) return 2;
    int rc = 0;
    for (int t = 0; t < nsteps && rc == 0; ++t) {
        rc = oracle_step(nx, ny, nz, tau, G, g, mask, f, tmp);
        memcpy(f, tmp, sizeof(double) * 2 * Q * N);
    }
    free(tmp);
    return rc;
}

/* Output moments: rho^k (C1) and the half-force-corrected mixture velocity
 * u = (sum_k sum_i c_i f_i^k + F_total/2) / rho; 0 at solid nodes. */
void oracle_moments(int nx, int ny, int nz, double G, const double* g,
                    const uint8_t* mask, const double* f,
                    double* rhoA, double* rhoB, double* u)
{
    lattice_setup();
    const long N = (long)nx * ny * nz;
    double* rho = (double*)malloc(sizeof(double) * 2 * N);
    double* F = (double*)malloc(sizeof(double) * 6 * N);
    if (!rho || !F) { free(rho); free(F); return; }
    oracle_density_force(nx, ny, nz, G, g, mask, f, rho, F);
    #pragma omp parallel for schedule(static)
    for (long s = 0; s < N; ++s) {
        rhoA[s] = rho[s];
        rhoB[s] = rho[N + s];
        if (!u) continue;
        double r = rho[s] + rho[N + s];
        for (int a = 0; a < 3; ++a) {
            double m = 0.0;
            for (int k = 0; k < 2; ++k)
                for (int i = 0; i < Q; ++i) m += CV[i][a] * f[(k*Q + i)*N + s];
            m += 0.5 * (F[(0*3 + a)*N + s] + F[(1*3 + a)*N + s]);
            u[a*N + s] = (is_fluid(mask, s) && r > 0.0) ? m / r : 0.0;
        }
    }
    free(rho); free(F);
}

/* Conserved totals over fluid nodes, summed serially in site order:
 * out[0] = sum rho^A, out[1] = sum rho^B, out[2..4] = sum_k sum_i c_i f_i^k. */
void oracle_stats(int nx, int ny, int nz, const uint8_t* mask, const double* f, double out[5])
{
    lattice_setup();
    const long N = (long)nx * ny * nz;
    for (int j = 0; j < 5; ++j) out[j] = 0.0;
    for (long s = 0; s < N; ++s) {
        if (!is_fluid(mask, s)) continue;
        for (int k = 0; k < 2; ++k)
            for (int i = 0; i < Q; ++i) {
                double v = f[(k*Q + i)*N + s];
                out[k] += v;
                for (int a = 0; a < 3; ++a) out[2 + a] += CV[i][a] * v;
            }
    }
}
