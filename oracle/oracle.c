/*
 * oracle.c -- plain, slow, single-threaded CPU reference (IEEE FP64) for
 * explicit time stepping of du/dt = F(t,u), u(0) = u0 (paper, Introduction).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may include, link,
 * load or call this file: only the tests, the smoke check and the benchmark's
 * CPU-baseline leg use it.  It shares no code with the CUDA library.
 *
 * Build: gcc -O2 -ffp-contract=off -fopenmp -fPIC -shared (no fast-math, no
 * FMA contraction), so every operation below is one correctly rounded IEEE op
 * in the order written.  The loops over cells and elements may be shared
 * among threads (orc_set_threads; 1 by default): each element's operations
 * and their order are the same whatever the thread count, and the only
 * reduction (the error norm's maximum) stays sequential.
 *
 * Contents, each following the passage cited at its definition:
 *   - right-hand sides: the Gray-Scott system (Eq. 2, read with the System
 *     functor of Listing 2 for the v-equation) on a periodic grid with the
 *     7-point central Laplacian; pointwise ODEs dx/dt = -x and x(1-x); the
 *     paper's exponential (Eq. 1a) and sigmoidal (Eq. 1b) families.
 *   - explicit Runge-Kutta steppers of Table 1 (explicit Euler, modified
 *     midpoint, RK4, Dormand-Prince 5 with its embedded order-4 solution), as one generic
 *     Butcher-tableau step: k_i = F(t + c_i dt, u + dt sum_j a_ij k_j),
 *     u_new = u + dt sum_i b_i k_i, err = dt sum_i (b_i - bhat_i) k_i.
 *   - the error-controlled adaptive driver (section "Architecture and
 *     nomenclature of Boost Odeint": error stepper + L-infinity norm + step
 *     size controller).  The paper gives no controller formula; the reading
 *     used here is stated at orc_integrate_adaptive.
 *   - the Adams-Bashforth 4 multistep method (Table 1) started by RK4, and
 *     Adams-Bashforth with 1..8 steps (Table 1, Fig. 2c,d) with coefficients
 *     integrated from their definition; Adams-Bashforth-Moulton with 1..8
 *     steps (Table 1) as an Adams-Bashforth predictor and an Adams-Moulton
 *     corrector (PECE), the weights likewise from their definition.
 *   - the further tableaux of Table 1: Cash-Karp 5(4) and Fehlberg 7(8), and
 *     the adaptive driver for any embedded pair; per-element adaptive
 *     integration of independent scalar ODEs (each its own step size).
 *   - the n-ary stage algebra y = sum_j a_j x_j (section "The distributed
 *     OpenFPM state type and algebra", for_each operations, up to 15 terms).
 *   - the DC-PSE Laplacian (section on the Gray-Scott benchmark, which cites
 *     Schrader et al.'s discretization-corrected PSE) on the regular grid, and
 *     the Gray-Scott right-hand side with it.
 *   - 3D periodic convolution forward / input-gradient / weight-gradient for
 *     the learned surrogate, by their definitions (plain loops).
 */
#include <math.h>
#include <omp.h>
#include <stdlib.h>
#include <string.h>

/* Threads for the cell / element loops (1 unless set). */
static int orc_threads = 1;
void orc_set_threads(int n) { orc_threads = n < 1 ? 1 : n; }
int orc_get_threads(void) { return orc_threads; }
int orc_max_threads(void) { return omp_get_num_procs(); }

/* ------------------------------------------------------------------------ */
/* Butcher tableaux (Table 1).  a is s x s row-major, strictly lower.        */
/* ------------------------------------------------------------------------ */

typedef struct {
    int s;
    double a[13 * 13];
    double b[13];
    double bhat[13]; /* embedded lower-order weights; valid if has_bhat */
    double c[13];
    int has_bhat;
} orc_tableau;

enum { ORC_EULER = 0, ORC_RK4 = 1, ORC_DOPRI5 = 2, ORC_CK54 = 3, ORC_RKF78 = 4, ORC_MIDPOINT = 5 };

/* Fills tableau T for method id; returns 0 on success. */
int orc_get_tableau(int id, orc_tableau* T) {
    memset(T, 0, sizeof(*T));
    if (id == ORC_EULER) {
        /* explicit Euler: one stage, b = 1 */
        T->s = 1;
        T->b[0] = 1.0;
        T->c[0] = 0.0;
        return 0;
    }
    if (id == ORC_MIDPOINT) {
        /* modified midpoint (Table 1, order 2) with two substeps of h = dt/2
         * (this build's reading of the substep count): z1 = y + h f(y),
         * z2 = y + 2h f(z1), y_new = (z1 + z2 + h f(z2)) / 2, written as the
         * tableau c = (0, 1/2, 1), a21 = 1/2, a32 = 1, b = (1/4, 1/2, 1/4) */
        T->s = 3;
        T->a[1 * 3 + 0] = 0.5;
        T->a[2 * 3 + 1] = 1.0;
        T->b[0] = 0.25; T->b[1] = 0.5; T->b[2] = 0.25;
        T->c[0] = 0.0; T->c[1] = 0.5; T->c[2] = 1.0;
        return 0;
    }
    if (id == ORC_RK4) {
        /* classical Runge-Kutta 4: c = (0, 1/2, 1/2, 1), b = (1,2,2,1)/6 */
        T->s = 4;
        T->a[1 * 4 + 0] = 0.5;
        T->a[2 * 4 + 1] = 0.5;
        T->a[3 * 4 + 2] = 1.0;
        T->b[0] = 1.0 / 6.0; T->b[1] = 1.0 / 3.0; T->b[2] = 1.0 / 3.0; T->b[3] = 1.0 / 6.0;
        T->c[0] = 0.0; T->c[1] = 0.5; T->c[2] = 0.5; T->c[3] = 1.0;
        return 0;
    }
    if (id == ORC_DOPRI5) {
        /* Dormand & Prince (1980) RK5(4)7M.  Row 7 equals b (first same as
         * last); bhat is the embedded order-4 solution. */
        const int s = 7;
        double* a = T->a;
        T->s = s;
        T->c[0] = 0.0; T->c[1] = 1.0 / 5.0; T->c[2] = 3.0 / 10.0; T->c[3] = 4.0 / 5.0;
        T->c[4] = 8.0 / 9.0; T->c[5] = 1.0; T->c[6] = 1.0;
        a[1 * s + 0] = 1.0 / 5.0;
        a[2 * s + 0] = 3.0 / 40.0;        a[2 * s + 1] = 9.0 / 40.0;
        a[3 * s + 0] = 44.0 / 45.0;       a[3 * s + 1] = -56.0 / 15.0;    a[3 * s + 2] = 32.0 / 9.0;
        a[4 * s + 0] = 19372.0 / 6561.0;  a[4 * s + 1] = -25360.0 / 2187.0;
        a[4 * s + 2] = 64448.0 / 6561.0;  a[4 * s + 3] = -212.0 / 729.0;
        a[5 * s + 0] = 9017.0 / 3168.0;   a[5 * s + 1] = -355.0 / 33.0;   a[5 * s + 2] = 46732.0 / 5247.0;
        a[5 * s + 3] = 49.0 / 176.0;      a[5 * s + 4] = -5103.0 / 18656.0;
        a[6 * s + 0] = 35.0 / 384.0;      a[6 * s + 1] = 0.0;             a[6 * s + 2] = 500.0 / 1113.0;
        a[6 * s + 3] = 125.0 / 192.0;     a[6 * s + 4] = -2187.0 / 6784.0; a[6 * s + 5] = 11.0 / 84.0;
        T->b[0] = 35.0 / 384.0; T->b[1] = 0.0; T->b[2] = 500.0 / 1113.0; T->b[3] = 125.0 / 192.0;
        T->b[4] = -2187.0 / 6784.0; T->b[5] = 11.0 / 84.0; T->b[6] = 0.0;
        T->bhat[0] = 5179.0 / 57600.0; T->bhat[1] = 0.0; T->bhat[2] = 7571.0 / 16695.0;
        T->bhat[3] = 393.0 / 640.0; T->bhat[4] = -92097.0 / 339200.0; T->bhat[5] = 187.0 / 2100.0;
        T->bhat[6] = 1.0 / 40.0;
        T->has_bhat = 1;
        return 0;
    }
    if (id == ORC_CK54) {
        /* Cash & Karp (1990) embedded 5(4): the order-5 solution b is
         * propagated, bhat is the order-4 one. */
        const int s = 6;
        double* a = T->a;
        T->s = s;
        T->c[0] = 0.0; T->c[1] = 1.0 / 5.0; T->c[2] = 3.0 / 10.0; T->c[3] = 3.0 / 5.0;
        T->c[4] = 1.0; T->c[5] = 7.0 / 8.0;
        a[1 * s + 0] = 1.0 / 5.0;
        a[2 * s + 0] = 3.0 / 40.0;         a[2 * s + 1] = 9.0 / 40.0;
        a[3 * s + 0] = 3.0 / 10.0;         a[3 * s + 1] = -9.0 / 10.0;     a[3 * s + 2] = 6.0 / 5.0;
        a[4 * s + 0] = -11.0 / 54.0;       a[4 * s + 1] = 5.0 / 2.0;       a[4 * s + 2] = -70.0 / 27.0;
        a[4 * s + 3] = 35.0 / 27.0;
        a[5 * s + 0] = 1631.0 / 55296.0;   a[5 * s + 1] = 175.0 / 512.0;   a[5 * s + 2] = 575.0 / 13824.0;
        a[5 * s + 3] = 44275.0 / 110592.0; a[5 * s + 4] = 253.0 / 4096.0;
        T->b[0] = 37.0 / 378.0; T->b[2] = 250.0 / 621.0; T->b[3] = 125.0 / 594.0; T->b[5] = 512.0 / 1771.0;
        T->bhat[0] = 2825.0 / 27648.0; T->bhat[2] = 18575.0 / 48384.0; T->bhat[3] = 13525.0 / 55296.0;
        T->bhat[4] = 277.0 / 14336.0;  T->bhat[5] = 1.0 / 4.0;
        T->has_bhat = 1;
        return 0;
    }
    if (id == ORC_RKF78) {
        /* Fehlberg (1968) embedded 7(8), 13 stages.  Table 1 lists the method
         * as order 8: the order-8 solution b is propagated, bhat is the order-7
         * one (they differ only in k1, k11, k12, k13). */
        const int s = 13;
        double* a = T->a;
        T->s = s;
        const double c[13] = {0.0, 2.0 / 27.0, 1.0 / 9.0, 1.0 / 6.0, 5.0 / 12.0, 1.0 / 2.0, 5.0 / 6.0,
                              1.0 / 6.0, 2.0 / 3.0, 1.0 / 3.0, 1.0, 0.0, 1.0};
        for (int i = 0; i < s; ++i) T->c[i] = c[i];
        a[1 * s + 0] = 2.0 / 27.0;
        a[2 * s + 0] = 1.0 / 36.0;      a[2 * s + 1] = 1.0 / 12.0;
        a[3 * s + 0] = 1.0 / 24.0;      a[3 * s + 2] = 1.0 / 8.0;
        a[4 * s + 0] = 5.0 / 12.0;      a[4 * s + 2] = -25.0 / 16.0;    a[4 * s + 3] = 25.0 / 16.0;
        a[5 * s + 0] = 1.0 / 20.0;      a[5 * s + 3] = 1.0 / 4.0;       a[5 * s + 4] = 1.0 / 5.0;
        a[6 * s + 0] = -25.0 / 108.0;   a[6 * s + 3] = 125.0 / 108.0;   a[6 * s + 4] = -65.0 / 27.0;
        a[6 * s + 5] = 125.0 / 54.0;
        a[7 * s + 0] = 31.0 / 300.0;    a[7 * s + 4] = 61.0 / 225.0;    a[7 * s + 5] = -2.0 / 9.0;
        a[7 * s + 6] = 13.0 / 900.0;
        a[8 * s + 0] = 2.0;             a[8 * s + 3] = -53.0 / 6.0;     a[8 * s + 4] = 704.0 / 45.0;
        a[8 * s + 5] = -107.0 / 9.0;    a[8 * s + 6] = 67.0 / 90.0;     a[8 * s + 7] = 3.0;
        a[9 * s + 0] = -91.0 / 108.0;   a[9 * s + 3] = 23.0 / 108.0;    a[9 * s + 4] = -976.0 / 135.0;
        a[9 * s + 5] = 311.0 / 54.0;    a[9 * s + 6] = -19.0 / 60.0;    a[9 * s + 7] = 17.0 / 6.0;
        a[9 * s + 8] = -1.0 / 12.0;
        a[10 * s + 0] = 2383.0 / 4100.0; a[10 * s + 3] = -341.0 / 164.0; a[10 * s + 4] = 4496.0 / 1025.0;
        a[10 * s + 5] = -301.0 / 82.0;   a[10 * s + 6] = 2133.0 / 4100.0; a[10 * s + 7] = 45.0 / 82.0;
        a[10 * s + 8] = 45.0 / 164.0;    a[10 * s + 9] = 18.0 / 41.0;
        a[11 * s + 0] = 3.0 / 205.0;     a[11 * s + 5] = -6.0 / 41.0;    a[11 * s + 6] = -3.0 / 205.0;
        a[11 * s + 7] = -3.0 / 41.0;     a[11 * s + 8] = 3.0 / 41.0;     a[11 * s + 9] = 6.0 / 41.0;
        a[12 * s + 0] = -1777.0 / 4100.0; a[12 * s + 3] = -341.0 / 164.0; a[12 * s + 4] = 4496.0 / 1025.0;
        a[12 * s + 5] = -289.0 / 82.0;   a[12 * s + 6] = 2193.0 / 4100.0; a[12 * s + 7] = 51.0 / 82.0;
        a[12 * s + 8] = 33.0 / 164.0;    a[12 * s + 9] = 12.0 / 41.0;    a[12 * s + 11] = 1.0;
        const double w7[13] = {41.0 / 840.0, 0, 0, 0, 0, 34.0 / 105.0, 9.0 / 35.0, 9.0 / 35.0, 9.0 / 280.0,
                               9.0 / 280.0, 41.0 / 840.0, 0, 0};
        const double w8[13] = {0, 0, 0, 0, 0, 34.0 / 105.0, 9.0 / 35.0, 9.0 / 35.0, 9.0 / 280.0,
                               9.0 / 280.0, 0, 41.0 / 840.0, 41.0 / 840.0};
        for (int i = 0; i < s; ++i) {
            T->b[i] = w8[i];
            T->bhat[i] = w7[i];
        }
        T->has_bhat = 1;
        return 0;
    }
    return 1;
}

/* Orders of an embedded pair for the step-size controller: p of the
 * propagated solution, q of the embedded one (0 if the method has none). */
int orc_pair_orders(int id, int* p, int* q) {
    switch (id) {
        case ORC_DOPRI5: *p = 5; *q = 4; return 0;
        case ORC_CK54: *p = 5; *q = 4; return 0;
        case ORC_RKF78: *p = 8; *q = 7; return 0;
        default: *p = 0; *q = 0; return 1;
    }
}

/* ------------------------------------------------------------------------ */
/* Right-hand sides F(t, y)                                                  */
/* ------------------------------------------------------------------------ */

typedef void (*orc_rhs_fn)(const void* sys, double t, long n, const double* y, double* f);

/* Gray-Scott system (Eq. 2 with the v-equation of Listing 2):
 *   du/dt = Du Lap(u) - u v^2 + F (1 - u)
 *   dv/dt = Dv Lap(v) + u v^2 - (F + k) v
 * on an nx*ny*nz periodic grid, spacing h_d = L_d / n_d, and the 7-point
 * central Laplacian Lap(w)_i = sum_d (w_{i+e_d} - 2 w_i + w_{i-e_d}) / h_d^2.
 * State vector y = [u (N values); v (N values)], cell index x + nx (y + ny z). */
typedef struct {
    int nx, ny, nz;
    double Lx, Ly, Lz;
    double Du, Dv, F, k;
} orc_gs;

static double orc_lap(const orc_gs* p, const double* w, int x, int y, int z) {
    const int nx = p->nx, ny = p->ny, nz = p->nz;
    const double hx = p->Lx / nx, hy = p->Ly / ny, hz = p->Lz / nz;
    const int xm = (x + nx - 1) % nx, xp = (x + 1) % nx;
    const int ym = (y + ny - 1) % ny, yp = (y + 1) % ny;
    const int zm = (z + nz - 1) % nz, zp = (z + 1) % nz;
#define ORC_AT(X, Y, Z) w[(long)(X) + (long)nx * ((long)(Y) + (long)ny * (long)(Z))]
    const double c = ORC_AT(x, y, z);
    const double lx = (ORC_AT(xm, y, z) - 2.0 * c + ORC_AT(xp, y, z)) / (hx * hx);
    const double ly = (ORC_AT(x, ym, z) - 2.0 * c + ORC_AT(x, yp, z)) / (hy * hy);
    const double lz = (ORC_AT(x, y, zm) - 2.0 * c + ORC_AT(x, y, zp)) / (hz * hz);
#undef ORC_AT
    return lx + ly + lz;
}

/* Lap(w) for a whole field (exported for the Laplacian pins). */
void orc_gs_laplacian(const orc_gs* p, const double* w, double* out) {
    #pragma omp parallel for num_threads(orc_threads) schedule(static) if ((long)p->nx * p->ny * p->nz >= 4096)
    for (int z = 0; z < p->nz; ++z)
        for (int y = 0; y < p->ny; ++y)
            for (int x = 0; x < p->nx; ++x)
                out[(long)x + (long)p->nx * ((long)y + (long)p->ny * z)] = orc_lap(p, w, x, y, z);
}

void orc_gs_rhs(const void* sys, double t, long n, const double* y, double* f) {
    (void)t;
    const orc_gs* p = (const orc_gs*)sys;
    const long N = (long)p->nx * p->ny * p->nz;
    (void)n; /* n == 2N */
    const double* u = y;
    const double* v = y + N;
    #pragma omp parallel for num_threads(orc_threads) schedule(static) if ((long)p->nx * p->ny * p->nz >= 4096)
    for (int z = 0; z < p->nz; ++z)
        for (int yy = 0; yy < p->ny; ++yy)
            for (int x = 0; x < p->nx; ++x) {
                const long i = (long)x + (long)p->nx * ((long)yy + (long)p->ny * z);
                const double uvv = u[i] * v[i] * v[i];
                f[i] = p->Du * orc_lap(p, u, x, yy, z) - uvv + p->F * (1.0 - u[i]);
                f[N + i] = p->Dv * orc_lap(p, v, x, yy, z) + uvv - (p->F + p->k) * v[i];
            }
}

/* Pointwise families.  kind 0: dx/dt = -x.  kind 1: dx/dt = x (1 - x).
 * kind 2: the exponential family of Eq. 1a, du/dt = c_i e^t, c_i = x_i y_i
 * given per element in coef.  kind 3: the sigmoidal family of Eq. 1b,
 * du/dt = s(t) (1 - s(t)), s(t) = 1 / (1 + e^-t). */
/* ------------------------------------------------------------------------ */
/* DC-PSE Laplacian on the regular grid.                                      */
/*                                                                            */
/* Discretization-corrected PSE (the operator the paper's Gray-Scott run      */
/* uses): for a derivative D^beta with |beta| = 2,                            */
/*   D^beta f(x_p) ~ eps^-2 sum_q (f(x_q) - f(x_p)) eta(z_q),                 */
/*   z_q = (x_p - x_q) / eps,  eta(z) = sum_g a_g z^alpha_g exp(-|z|^2),      */
/* over the neighbours q with |x_q - x_p| <= r_c, where the coefficients a_g  */
/* make the discrete moments of the kernel match those of the derivative:     */
/*   sum_q z_q^alpha eta(z_q) = (-1)^|alpha| alpha! delta_{alpha beta}        */
/* for every alpha with 1 <= |alpha| <= |beta| + r - 1 (convergence order r). */
/* The paper gives no kernel parameters; this build's reading: Gaussian        */
/* kernel, eps_d = h_d per axis (so z_q is the integer offset, negated),      */
/* r = 2 (|alpha| <= 3: 19 monomials), r_c = rc_over_h grid spacings.         */
/* The Laplacian is the sum over the three axes of the beta = 2 e_d operators; */
/* on a regular grid every point has the same neighbourhood, so the operator  */
/* is one stencil: L f_p = sum_q w_q (f_q - f_p).                            */
/* ------------------------------------------------------------------------ */
#define ORC_DCPSE_MAX 2048
typedef struct {
    int count;
    int off[ORC_DCPSE_MAX][3];
    double w[ORC_DCPSE_MAX];
} orc_dcpse;

static double orc_ipow(double x, int e) {
    double r = 1.0;
    for (int i = 0; i < e; ++i) r *= x;
    return r;
}

/* Solves the n x n system M a = b (row-major M, overwritten) by Gaussian
 * elimination with partial pivoting; returns 0 on success. */
static int orc_solve(int n, double* M, double* b, double* a) {
    for (int c = 0; c < n; ++c) {
        int piv = c;
        for (int r = c + 1; r < n; ++r)
            if (fabs(M[r * n + c]) > fabs(M[piv * n + c])) piv = r;
        if (M[piv * n + c] == 0.0) return 1;
        if (piv != c) {
            for (int k = 0; k < n; ++k) {
                const double t = M[c * n + k]; M[c * n + k] = M[piv * n + k]; M[piv * n + k] = t;
            }
            const double t = b[c]; b[c] = b[piv]; b[piv] = t;
        }
        for (int r = c + 1; r < n; ++r) {
            const double f = M[r * n + c] / M[c * n + c];
            for (int k = c; k < n; ++k) M[r * n + k] -= f * M[c * n + k];
            b[r] -= f * b[c];
        }
    }
    for (int r = n - 1; r >= 0; --r) {
        double acc = b[r];
        for (int k = r + 1; k < n; ++k) acc -= M[r * n + k] * a[k];
        a[r] = acc / M[r * n + r];
    }
    return 0;
}

int orc_dcpse_laplacian(double hx, double hy, double hz, double rc_over_h, orc_dcpse* S) {
    /* monomials z^alpha with 1 <= |alpha| <= 3 */
    int mono[19][3], nm = 0;
    for (int deg = 1; deg <= 3; ++deg)
        for (int a0 = deg; a0 >= 0; --a0)
            for (int a1 = deg - a0; a1 >= 0; --a1) {
                mono[nm][0] = a0; mono[nm][1] = a1; mono[nm][2] = deg - a0 - a1;
                ++nm;
            }
    /* neighbours: integer offsets o != 0 with |o| <= r_c (in spacings) */
    const int R = (int)floor(rc_over_h);
    S->count = 0;
    for (int dz = -R; dz <= R; ++dz)
        for (int dy = -R; dy <= R; ++dy)
            for (int dx = -R; dx <= R; ++dx) {
                if (dx == 0 && dy == 0 && dz == 0) continue;
                if ((double)(dx * dx + dy * dy + dz * dz) > rc_over_h * rc_over_h) continue;
                if (S->count >= ORC_DCPSE_MAX) return 1;
                S->off[S->count][0] = dx; S->off[S->count][1] = dy; S->off[S->count][2] = dz;
                S->w[S->count] = 0.0;
                ++S->count;
            }
    if (S->count < nm) return 1;
    const double h2[3] = {hx * hx, hy * hy, hz * hz};
    for (int d = 0; d < 3; ++d) {
        double M[19 * 19], b[19], a[19];
        for (int i = 0; i < nm; ++i) {
            b[i] = (mono[i][d] == 2 && mono[i][0] + mono[i][1] + mono[i][2] == 2) ? 2.0 : 0.0;
            for (int j = 0; j < nm; ++j) M[i * nm + j] = 0.0;
        }
        for (int q = 0; q < S->count; ++q) {
            const double z[3] = {-(double)S->off[q][0], -(double)S->off[q][1], -(double)S->off[q][2]};
            const double g = exp(-(z[0] * z[0] + z[1] * z[1] + z[2] * z[2]));
            double phi[19];
            for (int i = 0; i < nm; ++i)
                phi[i] = orc_ipow(z[0], mono[i][0]) * orc_ipow(z[1], mono[i][1]) * orc_ipow(z[2], mono[i][2]);
            for (int i = 0; i < nm; ++i)
                for (int j = 0; j < nm; ++j) M[i * nm + j] += phi[i] * phi[j] * g;
        }
        if (orc_solve(nm, M, b, a)) return 1;
        for (int q = 0; q < S->count; ++q) {
            const double z[3] = {-(double)S->off[q][0], -(double)S->off[q][1], -(double)S->off[q][2]};
            const double g = exp(-(z[0] * z[0] + z[1] * z[1] + z[2] * z[2]));
            double eta = 0.0;
            for (int i = 0; i < nm; ++i)
                eta += a[i] * orc_ipow(z[0], mono[i][0]) * orc_ipow(z[1], mono[i][1]) * orc_ipow(z[2], mono[i][2]);
            S->w[q] += eta * g / h2[d];
        }
    }
    return 0;
}

/* the DC-PSE Laplacian of a periodic field w at cell (x, y, z) */
static double orc_lap_dcpse(const orc_gs* p, const orc_dcpse* S, const double* w, int x, int y, int z) {
    const int nx = p->nx, ny = p->ny, nz = p->nz;
    const double c = w[(long)x + (long)nx * ((long)y + (long)ny * z)];
    double acc = 0.0;
    for (int q = 0; q < S->count; ++q) {
        const int X = ((x + S->off[q][0]) % nx + nx) % nx;
        const int Y = ((y + S->off[q][1]) % ny + ny) % ny;
        const int Z = ((z + S->off[q][2]) % nz + nz) % nz;
        acc += S->w[q] * (w[(long)X + (long)nx * ((long)Y + (long)ny * Z)] - c);
    }
    return acc;
}

typedef struct {
    orc_gs gs;
    const orc_dcpse* S;
} orc_gs_dcpse;

/* Gray-Scott (Eq. 2, v-equation of Listing 2) with the DC-PSE Laplacian. */
void orc_gs_rhs_dcpse(const void* sys, double t, long n, const double* y, double* f) {
    (void)t;
    (void)n;
    const orc_gs_dcpse* P = (const orc_gs_dcpse*)sys;
    const orc_gs* p = &P->gs;
    const long N = (long)p->nx * p->ny * p->nz;
    const double* u = y;
    const double* v = y + N;
    #pragma omp parallel for num_threads(orc_threads) schedule(static) if ((long)p->nx * p->ny * p->nz >= 4096)
    for (int z = 0; z < p->nz; ++z)
        for (int yy = 0; yy < p->ny; ++yy)
            for (int x = 0; x < p->nx; ++x) {
                const long i = (long)x + (long)p->nx * ((long)yy + (long)p->ny * z);
                const double uvv = u[i] * v[i] * v[i];
                f[i] = p->Du * orc_lap_dcpse(p, P->S, u, x, yy, z) - uvv + p->F * (1.0 - u[i]);
                f[N + i] = p->Dv * orc_lap_dcpse(p, P->S, v, x, yy, z) + uvv - (p->F + p->k) * v[i];
            }
}

typedef struct {
    int kind;
    const double* coef;
} orc_pointwise;

void orc_pointwise_rhs(const void* sys, double t, long n, const double* y, double* f) {
    const orc_pointwise* p = (const orc_pointwise*)sys;
    for (long i = 0; i < n; ++i) {
        switch (p->kind) {
            case 0: f[i] = -y[i]; break;
            case 1: f[i] = y[i] * (1.0 - y[i]); break;
            case 2: f[i] = p->coef[i] * exp(t); break;
            default: {
                const double s = 1.0 / (1.0 + exp(-t));
                f[i] = s * (1.0 - s);
            }
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Stage algebra: y = sum_j a_j x_j over n elements (the for_each operations */
/* of the custom Algebra, up to 15 operands).                               */
/* ------------------------------------------------------------------------ */
int orc_axpy(long n, int nterms, const double* a, const double* const* x, double* y) {
    if (nterms < 1 || nterms > 15) return 1;
    for (long i = 0; i < n; ++i) {
        double s = 0.0;
        for (int j = 0; j < nterms; ++j) s += a[j] * x[j][i];
        y[i] = s;
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* One explicit Runge-Kutta step with tableau T.                              */
/*   k_i  = F(t + c_i dt, y + dt * sum_{j<i} a_ij k_j)                        */
/*   yout = y + dt * sum_i b_i k_i                                            */
/*   err  = dt * sum_i (b_i - bhat_i) k_i        (if err != NULL)             */
/* k: s*n scratch (k_i at k + i*n), ytmp: n scratch.  yout may alias y.      */
/* ------------------------------------------------------------------------ */
/* The three element loops of a step, over elements [lo, hi). */
static void orc_stage_input(const orc_tableau* T, int i, long n, double dt, const double* y, const double* k,
                            double* ytmp, long lo, long hi) {
    const int s = T->s;
    for (long e = lo; e < hi; ++e) {
        double acc = 0.0;
        for (int j = 0; j < i; ++j) acc += T->a[i * s + j] * k[(long)j * n + e];
        ytmp[e] = y[e] + dt * acc;
    }
}
static void orc_step_error(const orc_tableau* T, long n, double dt, const double* k, double* err, long lo,
                           long hi) {
    const int s = T->s;
    for (long e = lo; e < hi; ++e) {
        double acc = 0.0;
        for (int i = 0; i < s; ++i) acc += (T->b[i] - T->bhat[i]) * k[(long)i * n + e];
        err[e] = dt * acc;
    }
}
static void orc_step_output(const orc_tableau* T, long n, double dt, const double* y, const double* k,
                            double* yout, long lo, long hi) {
    const int s = T->s;
    for (long e = lo; e < hi; ++e) {
        double acc = 0.0;
        for (int i = 0; i < s; ++i) acc += T->b[i] * k[(long)i * n + e];
        yout[e] = y[e] + dt * acc;
    }
}

/* Runs body(lo, hi) over [0, n): on the calling thread for small n or one
 * thread, else in contiguous blocks on orc_threads threads (each element is
 * processed once, by the same operations, in any case). */
#define ORC_FOR_ELEMENTS(n, CALL)                                                   \
    do {                                                                            \
        if ((n) < 4096 || orc_threads < 2) {                                        \
            const long lo = 0, hi = (n);                                            \
            CALL;                                                                   \
        } else {                                                                    \
            const long nb_ = 8L * orc_threads, sz_ = ((n) + nb_ - 1) / nb_;         \
            _Pragma("omp parallel for num_threads(orc_threads) schedule(static)")  \
            for (long b_ = 0; b_ < nb_; ++b_) {                                     \
                const long lo = b_ * sz_, hi = lo + sz_ < (n) ? lo + sz_ : (n);     \
                if (lo < hi) CALL;                                                  \
            }                                                                       \
        }                                                                           \
    } while (0)

void orc_rk_step(const orc_tableau* T, orc_rhs_fn F, const void* sys, long n, double t, double dt,
                 const double* y, double* yout, double* err, double* k, double* ytmp) {
    const int s = T->s;
    for (int i = 0; i < s; ++i) {
        ORC_FOR_ELEMENTS(n, orc_stage_input(T, i, n, dt, y, k, ytmp, lo, hi));
        F(sys, t + T->c[i] * dt, n, ytmp, k + (long)i * n);
    }
    if (err) ORC_FOR_ELEMENTS(n, orc_step_error(T, n, dt, k, err, lo, hi));
    ORC_FOR_ELEMENTS(n, orc_step_output(T, n, dt, y, k, yout, lo, hi));
}

/* integrate_const (Listing 3): nsteps fixed steps, t_m = t0 + m dt. */
int orc_integrate_const(int method, orc_rhs_fn F, const void* sys, long n, double* y, double t0,
                        double dt, long nsteps) {
    orc_tableau T;
    if (orc_get_tableau(method, &T)) return 1;
    double* k = (double*)malloc(sizeof(double) * (size_t)n * (size_t)T.s);
    double* ytmp = (double*)malloc(sizeof(double) * (size_t)n);
    if (!k || !ytmp) { free(k); free(ytmp); return 3; }
    for (long m = 0; m < nsteps; ++m)
        orc_rk_step(&T, F, sys, n, t0 + (double)m * dt, dt, y, y, NULL, k, ytmp);
    free(k);
    free(ytmp);
    return 0;
}

/* Fixed steps of a given dt sequence (replay of an adaptive run's accepted
 * steps): t advances by each dt in turn. */
int orc_integrate_replay(int method, orc_rhs_fn F, const void* sys, long n, double* y, double t0,
                         const double* dts, long nsteps) {
    orc_tableau T;
    if (orc_get_tableau(method, &T)) return 1;
    double* k = (double*)malloc(sizeof(double) * (size_t)n * (size_t)T.s);
    double* ytmp = (double*)malloc(sizeof(double) * (size_t)n);
    if (!k || !ytmp) { free(k); free(ytmp); return 3; }
    double t = t0;
    for (long m = 0; m < nsteps; ++m) {
        orc_rk_step(&T, F, sys, n, t, dts[m], y, y, NULL, k, ytmp);
        t += dts[m];
    }
    free(k);
    free(ytmp);
    return 0;
}

/* One error-stepper attempt: yout, and the scaled L-infinity error norm
 *   E = max_e |err_e| / (atol + rtol (|y_e| + dt |k1_e|))
 * (section "Architecture and nomenclature of Boost Odeint": the norm is
 * usually the L-infinity norm; the scaling by the state and its derivative
 * is this build's reading).  Returns E. */
double orc_error_attempt(const orc_tableau* T, orc_rhs_fn F, const void* sys, long n, double t,
                         double dt, const double* y, double* yout, double atol, double rtol,
                         double* err, double* k, double* ytmp) {
    orc_rk_step(T, F, sys, n, t, dt, y, yout, err, k, ytmp);
    double E = 0.0;
    for (long e = 0; e < n; ++e) {
        const double sc = atol + rtol * (fabs(y[e]) + dt * fabs(k[e]));
        const double r = fabs(err[e]) / sc;
        if (isnan(E)) continue;             /* a NaN ratio, once seen, stays */
        if (isnan(r) || r > E) E = r;
    }
    return E;
}

/* Status codes (same meaning as the library's). */
enum { ORC_OK = 0, ORC_ERR_INVALID = 1, ORC_ERR_NOMEM = 3, ORC_ERR_STEP_UNDERFLOW = 4,
       ORC_ERR_MAX_STEPS = 5, ORC_ERR_NONFINITE = 6 };

/* integrate_adaptive with an embedded pair (Dormand-Prince 5(4) by default;
 * Cash-Karp 5(4), Fehlberg 7(8)).
 *
 * The paper states only that adaptive steppers size each step from an error
 * estimate and a tolerance, with an L-infinity norm.  The controller read
 * here (propagated order p, embedded order q: Dormand-Prince and Cash-Karp
 * p = 5, q = 4; Fehlberg p = 8, q = 7):
 *   attempt size h = dt, clipped to t_end - t if t + dt >= t_end;
 *   E > 1            : reject; dt = h * max(0.9 E^(-1/(q-1)), 0.2)
 *   E < 0.5          : accept; dt = h * 0.9 * max(E, 5^-p)^(-1/p)
 *   0.5 <= E <= 1    : accept; dt = h
 *   E not finite     : stop with NONFINITE
 *   max_rej consecutive rejections, or t + h == t: stop with STEP_UNDERFLOW.
 * On accept t += h (t = t_end exactly on a clipped step).  The loop ends when
 * t reaches t_end or after max_acc accepted steps (max_acc < 0: no limit).
 * If log_dt != NULL the accepted step sizes are written there (up to log_cap).
 * The core also records every attempt (its size h, its norm E, whether it
 * was accepted) when given trace arrays: the controller pins replay that
 * record against the closed-form error of dx/dt = -x.
 */
static int orc_adaptive_core(int method, orc_rhs_fn F, const void* sys, long n, double* y, double* t_io,
                             double t_end, double* dt_io, double atol, double rtol, long max_acc,
                             long max_rej, long* n_acc_out, long* n_rej_out, double* log_dt,
                             long log_cap, double* trace_h, double* trace_E, int* trace_acc,
                             long trace_cap, long* n_trace) {
    orc_tableau T;
    int po = 0, qo = 0;
    if (orc_get_tableau(method, &T) || orc_pair_orders(method, &po, &qo)) return ORC_ERR_INVALID;
    const int s = T.s;
    double* k = (double*)malloc(sizeof(double) * (size_t)n * (size_t)s);
    double* ytmp = (double*)malloc(sizeof(double) * (size_t)n);
    double* ynew = (double*)malloc(sizeof(double) * (size_t)n);
    double* err = (double*)malloc(sizeof(double) * (size_t)n);
    if (!k || !ytmp || !ynew || !err) { free(k); free(ytmp); free(ynew); free(err); return ORC_ERR_NOMEM; }
    double t = *t_io, dt = *dt_io;
    long n_acc = 0, n_rej = 0, consec = 0, n_att = 0;
    int status = ORC_OK;
    while (t < t_end && (max_acc < 0 || n_acc < max_acc)) {
        int last = 0;
        double h = dt;
        if (t + dt >= t_end) { h = t_end - t; last = 1; }
        if (!(h > 0.0) || t + h == t) { status = ORC_ERR_STEP_UNDERFLOW; break; }
        const double E = orc_error_attempt(&T, F, sys, n, t, h, y, ynew, atol, rtol, err, k, ytmp);
        if (trace_h && n_att < trace_cap) {
            trace_h[n_att] = h;
            trace_E[n_att] = E;
            trace_acc[n_att] = isfinite(E) && E <= 1.0;
        }
        ++n_att;
        if (!isfinite(E)) { status = ORC_ERR_NONFINITE; break; }
        if (E > 1.0) {
            ++n_rej; ++consec;
            double fac = 0.9 * pow(E, -1.0 / (double)(qo - 1));
            if (fac < 0.2) fac = 0.2;
            dt = h * fac;
            if (consec >= max_rej) { status = ORC_ERR_STEP_UNDERFLOW; break; }
            continue;
        }
        consec = 0;
        memcpy(y, ynew, sizeof(double) * (size_t)n);
        if (log_dt && n_acc < log_cap) log_dt[n_acc] = h;
        ++n_acc;
        t = last ? t_end : t + h;
        if (E < 0.5) {
            double Em = E;
            const double floor5 = pow(5.0, -(double)po);
            if (Em < floor5) Em = floor5;
            dt = h * 0.9 * pow(Em, -1.0 / (double)po);
        } else {
            dt = h;
        }
    }
    *t_io = t;
    *dt_io = dt;
    if (n_acc_out) *n_acc_out = n_acc;
    if (n_rej_out) *n_rej_out = n_rej;
    if (n_trace) *n_trace = n_att;
    free(k); free(ytmp); free(ynew); free(err);
    return status;
}

int orc_integrate_adaptive_m(int method, orc_rhs_fn F, const void* sys, long n, double* y, double* t_io,
                             double t_end, double* dt_io, double atol, double rtol, long max_acc,
                             long max_rej, long* n_acc_out, long* n_rej_out, double* log_dt,
                             long log_cap) {
    return orc_adaptive_core(method, F, sys, n, y, t_io, t_end, dt_io, atol, rtol, max_acc, max_rej, n_acc_out,
                             n_rej_out, log_dt, log_cap, NULL, NULL, NULL, 0, NULL);
}

int orc_integrate_adaptive(orc_rhs_fn F, const void* sys, long n, double* y, double* t_io,
                           double t_end, double* dt_io, double atol, double rtol, long max_acc,
                           long max_rej, long* n_acc_out, long* n_rej_out, double* log_dt,
                           long log_cap) {
    return orc_integrate_adaptive_m(ORC_DOPRI5, F, sys, n, y, t_io, t_end, dt_io, atol, rtol, max_acc,
                                    max_rej, n_acc_out, n_rej_out, log_dt, log_cap);
}

/* Adams-Bashforth with s steps (Table 1: 1..8; Fig. 2c,d):
 *   u_{m+1} = u_m + dt sum_{j<s} beta_j f_{m-j},
 * beta_j = the integral over [t_m, t_m + dt] of the Lagrange basis polynomial
 * of node t_{m-j} among the nodes t_m, ..., t_{m-s+1}, divided by dt.  In
 * the unit variable tau (node m-j at tau = -j):
 *   beta_j = int_0^1 prod_{i != j} (tau + i) / (i - j) dtau.
 * The polynomial is expanded in powers of tau and integrated term by term. */
int orc_ab_coefficients(int s, double* beta) {
    if (s < 1 || s > 8) return ORC_ERR_INVALID;
    for (int j = 0; j < s; ++j) {
        double poly[9] = {1.0, 0, 0, 0, 0, 0, 0, 0, 0}; /* coefficients of tau^0..tau^8 */
        int deg = 0;
        double denom = 1.0;
        for (int i = 0; i < s; ++i) {
            if (i == j) continue;
            /* multiply by (tau + i) */
            for (int d = deg + 1; d >= 1; --d) poly[d] = poly[d - 1] + (double)i * poly[d];
            poly[0] = (double)i * poly[0];
            ++deg;
            denom *= (double)(i - j);
        }
        double integral = 0.0;
        for (int d = 0; d <= deg; ++d) integral += poly[d] / (double)(d + 1);
        beta[j] = integral / denom;
    }
    return ORC_OK;
}

/* Adams-Bashforth with s steps, t_m = t0 + m dt.  The first s - 1 steps of
 * a call are one-step steps of order >= s (this build's reading: the paper
 * does not say how the history is started): RK4 for s <= 4, the order-8
 * Fehlberg solution for s >= 5, so the start-up does not limit the observed
 * order.  s = 1 is explicit Euler. */
int orc_integrate_ab(int s, orc_rhs_fn F, const void* sys, long n, double* y, double t0, double dt,
                     long nsteps) {
    double beta[8];
    if (orc_ab_coefficients(s, beta)) return ORC_ERR_INVALID;
    orc_tableau T;
    orc_get_tableau(s <= 4 ? ORC_RK4 : ORC_RKF78, &T);
    double* f = (double*)malloc(sizeof(double) * (size_t)n * (size_t)s);
    double* k = (double*)malloc(sizeof(double) * (size_t)n * (size_t)T.s);
    double* ytmp = (double*)malloc(sizeof(double) * (size_t)n);
    if (!f || !k || !ytmp) { free(f); free(k); free(ytmp); return ORC_ERR_NOMEM; }
    double* fm[8];
    for (int j = 0; j < s; ++j) fm[j] = f + (long)j * n; /* fm[j] = f_{m-j} */
    for (long m = 0; m < nsteps; ++m) {
        const double t = t0 + (double)m * dt;
        double* oldest = fm[s - 1];
        for (int j = s - 1; j >= 1; --j) fm[j] = fm[j - 1];
        fm[0] = oldest;
        F(sys, t, n, y, fm[0]);
        if (m < s - 1) {
            orc_rk_step(&T, F, sys, n, t, dt, y, y, NULL, k, ytmp);
        } else {
            for (long e = 0; e < n; ++e) {
                double acc = 0.0;
                for (int j = 0; j < s; ++j) acc += beta[j] * fm[j][e];
                y[e] = y[e] + dt * acc;
            }
        }
    }
    free(f); free(k); free(ytmp);
    return ORC_OK;
}

/* Adams-Moulton weights with s nodes (the corrector of Table 1's
 * Adams-Bashforth-Moulton, s = 1..8):
 *   u_{m+1} = u_m + dt sum_{j<s} beta*_j f_{m+1-j},
 * beta*_j = the integral over [t_m, t_m + dt] of the Lagrange basis
 * polynomial of node t_{m+1-j} among t_{m+1}, t_m, ..., t_{m+2-s}, divided
 * by dt.  In the unit variable tau (node m+1-j at tau = 1 - j):
 *   beta*_j = int_0^1 prod_{i != j} (tau - 1 + i) / (i - j) dtau,
 * expanded in powers of tau and integrated term by term. */
int orc_am_coefficients(int s, double* beta) {
    if (s < 1 || s > 8) return ORC_ERR_INVALID;
    for (int j = 0; j < s; ++j) {
        double poly[9] = {1.0, 0, 0, 0, 0, 0, 0, 0, 0}; /* coefficients of tau^0..tau^8 */
        int deg = 0;
        double denom = 1.0;
        for (int i = 0; i < s; ++i) {
            if (i == j) continue;
            const double c = (double)(i - 1); /* multiply by (tau + c) */
            for (int d = deg + 1; d >= 1; --d) poly[d] = poly[d - 1] + c * poly[d];
            poly[0] = c * poly[0];
            ++deg;
            denom *= (double)(i - j);
        }
        double integral = 0.0;
        for (int d = 0; d <= deg; ++d) integral += poly[d] / (double)(d + 1);
        beta[j] = integral / denom;
    }
    return ORC_OK;
}

/* Adams-Bashforth-Moulton with s steps (Table 1: 1..8), as a
 * predictor-corrector in PECE form (this build's reading; the paper names
 * the method only): with f_m = F(t_m, u_m),
 *   predict   u* = u_m + dt sum_{j<s} beta_j f_{m-j}        (Adams-Bashforth)
 *   evaluate  f* = F(t_{m+1}, u*)
 *   correct   u_{m+1} = u_m + dt (beta*_0 f* + sum_{1<=j<s} beta*_j f_{m+1-j})
 *                                                            (Adams-Moulton)
 *   evaluate  f_{m+1} = F(t_{m+1}, u_{m+1}) at the next step's start.
 * t_m = t0 + m dt; the first s - 1 steps are one-step steps of order >= s,
 * as for Adams-Bashforth (RK4 for s <= 4, the order-8 Fehlberg solution
 * for s >= 5). */
int orc_integrate_abm(int s, orc_rhs_fn F, const void* sys, long n, double* y, double t0, double dt,
                      long nsteps) {
    double beta[8], betas[8];
    if (orc_ab_coefficients(s, beta) || orc_am_coefficients(s, betas)) return ORC_ERR_INVALID;
    orc_tableau T;
    orc_get_tableau(s <= 4 ? ORC_RK4 : ORC_RKF78, &T);
    double* f = (double*)malloc(sizeof(double) * (size_t)n * (size_t)s);
    double* k = (double*)malloc(sizeof(double) * (size_t)n * (size_t)T.s);
    double* ytmp = (double*)malloc(sizeof(double) * (size_t)n);
    double* fp = (double*)malloc(sizeof(double) * (size_t)n);
    if (!f || !k || !ytmp || !fp) { free(f); free(k); free(ytmp); free(fp); return ORC_ERR_NOMEM; }
    double* fm[8];
    for (int j = 0; j < s; ++j) fm[j] = f + (long)j * n; /* fm[j] = f_{m-j} */
    for (long m = 0; m < nsteps; ++m) {
        const double t = t0 + (double)m * dt;
        double* oldest = fm[s - 1];
        for (int j = s - 1; j >= 1; --j) fm[j] = fm[j - 1];
        fm[0] = oldest;
        F(sys, t, n, y, fm[0]);
        if (m < s - 1) {
            orc_rk_step(&T, F, sys, n, t, dt, y, y, NULL, k, ytmp);
            continue;
        }
        for (long e = 0; e < n; ++e) {
            double acc = 0.0;
            for (int j = 0; j < s; ++j) acc += beta[j] * fm[j][e];
            ytmp[e] = y[e] + dt * acc;
        }
        F(sys, t0 + (double)(m + 1) * dt, n, ytmp, fp);
        for (long e = 0; e < n; ++e) {
            double acc = betas[0] * fp[e];
            for (int j = 1; j < s; ++j) acc += betas[j] * fm[j - 1][e];
            y[e] = y[e] + dt * acc;
        }
    }
    free(f); free(k); free(ytmp); free(fp);
    return ORC_OK;
}

/* Adams-Bashforth 4 (Table 1, multi-step), started with three RK4 steps:
 *   u_{m+1} = u_m + dt/24 (55 f_m - 59 f_{m-1} + 37 f_{m-2} - 9 f_{m-3}),
 * f_m = F(t_m, u_m), t_m = t0 + m dt.  nsteps counts all steps, the RK4
 * start-up steps included. */
int orc_integrate_ab4(orc_rhs_fn F, const void* sys, long n, double* y, double t0, double dt,
                      long nsteps) {
    orc_tableau T;
    orc_get_tableau(ORC_RK4, &T);
    double* f = (double*)malloc(sizeof(double) * (size_t)n * 4); /* f_m, f_{m-1}, f_{m-2}, f_{m-3} */
    double* k = (double*)malloc(sizeof(double) * (size_t)n * 4);
    double* ytmp = (double*)malloc(sizeof(double) * (size_t)n);
    if (!f || !k || !ytmp) { free(f); free(k); free(ytmp); return ORC_ERR_NOMEM; }
    double* fm[4] = {f, f + n, f + 2 * n, f + 3 * n}; /* fm[j] = f_{m-j} */
    for (long m = 0; m < nsteps; ++m) {
        const double t = t0 + (double)m * dt;
        /* rotate history: f_{m-j} <- f_{m-j+1} */
        double* oldest = fm[3];
        fm[3] = fm[2]; fm[2] = fm[1]; fm[1] = fm[0]; fm[0] = oldest;
        F(sys, t, n, y, fm[0]);
        if (m < 3) {
            orc_rk_step(&T, F, sys, n, t, dt, y, y, NULL, k, ytmp);
        } else {
            for (long e = 0; e < n; ++e)
                y[e] = y[e] + dt / 24.0 * (55.0 * fm[0][e] - 59.0 * fm[1][e] + 37.0 * fm[2][e] -
                                           9.0 * fm[3][e]);
        }
    }
    free(f); free(k); free(ytmp);
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Convenience entry points with concrete systems (for ctypes).             */
/* ------------------------------------------------------------------------ */
void orc_gs_rhs_full(const orc_gs* p, const double* y, double* f) {
    orc_gs_rhs(p, 0.0, 2L * p->nx * p->ny * p->nz, y, f);
}
int orc_gs_integrate_const(const orc_gs* p, int method, double* y, double t0, double dt, long nsteps) {
    return orc_integrate_const(method, orc_gs_rhs, p, 2L * p->nx * p->ny * p->nz, y, t0, dt, nsteps);
}
int orc_gs_integrate_replay(const orc_gs* p, int method, double* y, double t0, const double* dts,
                            long nsteps) {
    return orc_integrate_replay(method, orc_gs_rhs, p, 2L * p->nx * p->ny * p->nz, y, t0, dts, nsteps);
}
int orc_gs_integrate_adaptive(const orc_gs* p, double* y, double* t, double t_end, double* dt,
                              double atol, double rtol, long max_acc, long max_rej, long* n_acc,
                              long* n_rej, double* log_dt, long log_cap) {
    return orc_integrate_adaptive(orc_gs_rhs, p, 2L * p->nx * p->ny * p->nz, y, t, t_end, dt, atol,
                                  rtol, max_acc, max_rej, n_acc, n_rej, log_dt, log_cap);
}
int orc_gs_integrate_adaptive_m(const orc_gs* p, int method, double* y, double* t, double t_end, double* dt,
                                double atol, double rtol, long max_acc, long max_rej, long* n_acc, long* n_rej,
                                double* log_dt, long log_cap) {
    return orc_integrate_adaptive_m(method, orc_gs_rhs, p, 2L * p->nx * p->ny * p->nz, y, t, t_end, dt, atol, rtol,
                                    max_acc, max_rej, n_acc, n_rej, log_dt, log_cap);
}
int orc_gs_integrate_ab4(const orc_gs* p, double* y, double t0, double dt, long nsteps) {
    return orc_integrate_ab4(orc_gs_rhs, p, 2L * p->nx * p->ny * p->nz, y, t0, dt, nsteps);
}
/* One Dopri5 attempt on the GS system: yout, err and the scaled norm. */
double orc_gs_dopri5_attempt(const orc_gs* p, double t, double dt, const double* y, double* yout,
                             double* err, double atol, double rtol) {
    orc_tableau T;
    orc_get_tableau(ORC_DOPRI5, &T);
    const long n = 2L * p->nx * p->ny * p->nz;
    double* k = (double*)malloc(sizeof(double) * (size_t)n * (size_t)T.s);
    double* ytmp = (double*)malloc(sizeof(double) * (size_t)n);
    double E = NAN;
    if (k && ytmp) E = orc_error_attempt(&T, orc_gs_rhs, p, n, t, dt, y, yout, atol, rtol, err, k, ytmp);
    free(k); free(ytmp);
    return E;
}

/* DC-PSE stencil of a grid (offsets in spacings, weights); returns the
 * neighbour count or -1. */
int orc_dcpse_stencil(double hx, double hy, double hz, double rc_over_h, int* off, double* w, int cap) {
    static orc_dcpse S;
    if (orc_dcpse_laplacian(hx, hy, hz, rc_over_h, &S) || S.count > cap) return -1;
    for (int q = 0; q < S.count; ++q) {
        off[3 * q] = S.off[q][0]; off[3 * q + 1] = S.off[q][1]; off[3 * q + 2] = S.off[q][2];
        w[q] = S.w[q];
    }
    return S.count;
}
int orc_gs_dcpse_rhs_full(const orc_gs* p, double rc_over_h, const double* y, double* f) {
    static orc_dcpse S;
    if (orc_dcpse_laplacian(p->Lx / p->nx, p->Ly / p->ny, p->Lz / p->nz, rc_over_h, &S)) return 1;
    orc_gs_dcpse P = {*p, &S};
    orc_gs_rhs_dcpse(&P, 0.0, 2L * p->nx * p->ny * p->nz, y, f);
    return 0;
}
int orc_gs_dcpse_integrate_const(const orc_gs* p, double rc_over_h, int method, double* y, double t0, double dt,
                                 long nsteps) {
    static orc_dcpse S;
    if (orc_dcpse_laplacian(p->Lx / p->nx, p->Ly / p->ny, p->Lz / p->nz, rc_over_h, &S)) return 1;
    orc_gs_dcpse P = {*p, &S};
    return orc_integrate_const(method, orc_gs_rhs_dcpse, &P, 2L * p->nx * p->ny * p->nz, y, t0, dt, nsteps);
}

int orc_gs_dcpse_integrate_adaptive_m(const orc_gs* p, double rc_over_h, int method, double* y, double* t,
                                      double t_end, double* dt, double atol, double rtol, long max_acc, long max_rej,
                                      long* n_acc, long* n_rej, double* log_dt, long log_cap) {
    static orc_dcpse S;
    if (orc_dcpse_laplacian(p->Lx / p->nx, p->Ly / p->ny, p->Lz / p->nz, rc_over_h, &S)) return ORC_ERR_INVALID;
    orc_gs_dcpse P = {*p, &S};
    return orc_integrate_adaptive_m(method, orc_gs_rhs_dcpse, &P, 2L * p->nx * p->ny * p->nz, y, t, t_end, dt, atol,
                                    rtol, max_acc, max_rej, n_acc, n_rej, log_dt, log_cap);
}
int orc_gs_dcpse_integrate_adaptive(const orc_gs* p, double rc_over_h, double* y, double* t, double t_end, double* dt,
                                    double atol, double rtol, long max_acc, long max_rej, long* n_acc, long* n_rej,
                                    double* log_dt, long log_cap) {
    return orc_gs_dcpse_integrate_adaptive_m(p, rc_over_h, ORC_DOPRI5, y, t, t_end, dt, atol, rtol, max_acc, max_rej,
                                             n_acc, n_rej, log_dt, log_cap);
}

void orc_pw_rhs(int kind, const double* coef, double t, long n, const double* y, double* f) {
    orc_pointwise p = {kind, coef};
    orc_pointwise_rhs(&p, t, n, y, f);
}
int orc_pw_integrate_const(int kind, const double* coef, int method, long n, double* y, double t0,
                           double dt, long nsteps) {
    orc_pointwise p = {kind, coef};
    return orc_integrate_const(method, orc_pointwise_rhs, &p, n, y, t0, dt, nsteps);
}
int orc_pw_integrate_replay(int kind, const double* coef, int method, long n, double* y, double t0,
                            const double* dts, long nsteps) {
    orc_pointwise p = {kind, coef};
    return orc_integrate_replay(method, orc_pointwise_rhs, &p, n, y, t0, dts, nsteps);
}
int orc_pw_integrate_adaptive(int kind, const double* coef, long n, double* y, double* t,
                              double t_end, double* dt, double atol, double rtol, long max_acc,
                              long max_rej, long* n_acc, long* n_rej, double* log_dt, long log_cap) {
    orc_pointwise p = {kind, coef};
    return orc_integrate_adaptive(orc_pointwise_rhs, &p, n, y, t, t_end, dt, atol, rtol, max_acc,
                                  max_rej, n_acc, n_rej, log_dt, log_cap);
}
int orc_pw_integrate_ab4(int kind, const double* coef, long n, double* y, double t0, double dt,
                         long nsteps) {
    orc_pointwise p = {kind, coef};
    return orc_integrate_ab4(orc_pointwise_rhs, &p, n, y, t0, dt, nsteps);
}
int orc_pw_integrate_ab(int steps, int kind, const double* coef, long n, double* y, double t0, double dt,
                        long nsteps) {
    orc_pointwise p = {kind, coef};
    return orc_integrate_ab(steps, orc_pointwise_rhs, &p, n, y, t0, dt, nsteps);
}
int orc_pw_integrate_abm(int steps, int kind, const double* coef, long n, double* y, double t0, double dt,
                         long nsteps) {
    orc_pointwise p = {kind, coef};
    return orc_integrate_abm(steps, orc_pointwise_rhs, &p, n, y, t0, dt, nsteps);
}
int orc_gs_integrate_abm(const orc_gs* p, int steps, double* y, double t0, double dt, long nsteps) {
    return orc_integrate_abm(steps, orc_gs_rhs, p, 2L * p->nx * p->ny * p->nz, y, t0, dt, nsteps);
}
int orc_pw_integrate_adaptive_m(int method, int kind, const double* coef, long n, double* y, double* t,
                                double t_end, double* dt, double atol, double rtol, long max_acc,
                                long max_rej, long* n_acc, long* n_rej, double* log_dt, long log_cap) {
    orc_pointwise p = {kind, coef};
    return orc_integrate_adaptive_m(method, orc_pointwise_rhs, &p, n, y, t, t_end, dt, atol, rtol, max_acc,
                                    max_rej, n_acc, n_rej, log_dt, log_cap);
}
/* orc_pw_integrate_adaptive_m with the record of every attempt: trace_h[a],
 * trace_E[a], trace_acc[a] for attempts a < min(*n_trace, trace_cap). */
int orc_pw_integrate_adaptive_trace(int method, int kind, const double* coef, long n, double* y, double* t,
                                    double t_end, double* dt, double atol, double rtol, long max_acc,
                                    long max_rej, long* n_acc, long* n_rej, double* trace_h, double* trace_E,
                                    int* trace_acc, long trace_cap, long* n_trace) {
    orc_pointwise p = {kind, coef};
    return orc_adaptive_core(method, orc_pointwise_rhs, &p, n, y, t, t_end, dt, atol, rtol, max_acc, max_rej,
                             n_acc, n_rej, NULL, 0, trace_h, trace_E, trace_acc, trace_cap, n_trace);
}
/* Independent scalar ODEs, each with its own step size and controller: the
 * adaptive driver applied to each element alone (element e: a one-element
 * system; its coefficient coef[e] for the Eq. 1a family).  Per-element
 * results: final t, next dt, accepted and rejected counts, status. */
int orc_pw_integrate_adaptive_each(int method, int kind, const double* coef, long n, double* y, double t0,
                                   double t_end, double dt0, double atol, double rtol, long max_acc,
                                   long max_rej, double* t_out, double* dt_out, long* n_acc, long* n_rej,
                                   int* status) {
#pragma omp parallel for num_threads(orc_threads) schedule(dynamic, 64)
    for (long e = 0; e < n; ++e) {
        orc_pointwise p = {kind, coef ? coef + e : NULL};
        double t = t0, dt = dt0;
        long na = 0, nr = 0;
        const int st = orc_integrate_adaptive_m(method, orc_pointwise_rhs, &p, 1, y + e, &t, t_end, &dt, atol,
                                                rtol, max_acc, max_rej, &na, &nr, NULL, 0);
        t_out[e] = t;
        dt_out[e] = dt;
        n_acc[e] = na;
        n_rej[e] = nr;
        status[e] = st;
    }
    for (long e = 0; e < n; ++e)
        if (status[e] == ORC_ERR_INVALID || status[e] == ORC_ERR_NOMEM) return status[e];
    return ORC_OK;
}
/* One Dopri5 attempt on a pointwise system: yout, err, returns the norm. */
double orc_pw_dopri5_attempt(int kind, const double* coef, long n, double t, double dt,
                             const double* y, double* yout, double* err, double atol, double rtol) {
    orc_pointwise p = {kind, coef};
    orc_tableau T;
    orc_get_tableau(ORC_DOPRI5, &T);
    double* k = (double*)malloc(sizeof(double) * (size_t)n * (size_t)T.s);
    double* ytmp = (double*)malloc(sizeof(double) * (size_t)n);
    double E = NAN;
    if (k && ytmp) E = orc_error_attempt(&T, orc_pointwise_rhs, &p, n, t, dt, y, yout, atol, rtol, err, k, ytmp);
    free(k); free(ytmp);
    return E;
}

/* ------------------------------------------------------------------------ */
/* 3D periodic convolution (learned surrogate), plain loops, FP64.          */
/* Activations: channels-last [D][H][W][C] with x = W fastest over cells.    */
/* Weights: [3][3][3][Cin][Cout] indexed by offsets (dz,dy,dx) in {-1,0,1}.  */
/*   y[z,y,x,o] = b[o] + sum_{dz,dy,dx,i} w[dz+1,dy+1,dx+1,i,o]              */
/*                                  * x[(z+dz)%D, (y+dy)%H, (x+dx)%W, i]     */
/* ------------------------------------------------------------------------ */
static long orc_wrap(long a, long n) { return ((a % n) + n) % n; }

void orc_conv3d_fwd(int D, int H, int W, int Cin, int Cout, const double* x, const double* w,
                    const double* b, double* y) {
    for (long z = 0; z < D; ++z)
        for (long yy = 0; yy < H; ++yy)
            for (long xx = 0; xx < W; ++xx)
                for (int o = 0; o < Cout; ++o) {
                    double acc = b ? b[o] : 0.0;
                    for (int dz = -1; dz <= 1; ++dz)
                        for (int dy = -1; dy <= 1; ++dy)
                            for (int dx = -1; dx <= 1; ++dx) {
                                const long zz = orc_wrap(z + dz, D), y2 = orc_wrap(yy + dy, H), x2 = orc_wrap(xx + dx, W);
                                const long tap = (long)((dz + 1) * 9 + (dy + 1) * 3 + (dx + 1));
                                for (int i = 0; i < Cin; ++i)
                                    acc += w[(tap * Cin + i) * Cout + o] *
                                           x[((zz * H + y2) * W + x2) * Cin + i];
                            }
                    y[((z * H + yy) * W + xx) * Cout + o] = acc;
                }
}

/* dL/dx given dL/dy: each input cell collects from the outputs it fed. */
void orc_conv3d_dgrad(int D, int H, int W, int Cin, int Cout, const double* dy, const double* w,
                      double* dx) {
    for (long z = 0; z < D; ++z)
        for (long yy = 0; yy < H; ++yy)
            for (long xx = 0; xx < W; ++xx)
                for (int i = 0; i < Cin; ++i) {
                    double acc = 0.0;
                    for (int dz = -1; dz <= 1; ++dz)
                        for (int dyo = -1; dyo <= 1; ++dyo)
                            for (int dxo = -1; dxo <= 1; ++dxo) {
                                /* output cell q = p - offset used input p at offset */
                                const long zz = orc_wrap(z - dz, D), y2 = orc_wrap(yy - dyo, H), x2 = orc_wrap(xx - dxo, W);
                                const long tap = (long)((dz + 1) * 9 + (dyo + 1) * 3 + (dxo + 1));
                                for (int o = 0; o < Cout; ++o)
                                    acc += w[(tap * Cin + i) * Cout + o] *
                                           dy[((zz * H + y2) * W + x2) * Cout + o];
                            }
                    dx[((z * H + yy) * W + xx) * Cin + i] = acc;
                }
}

/* dL/dw and dL/db given dL/dy (sums over all cells). */
void orc_conv3d_wgrad(int D, int H, int W, int Cin, int Cout, const double* x, const double* dy,
                      double* dw, double* db) {
    for (long tap = 0; tap < 27; ++tap) {
        const int dz = (int)(tap / 9) - 1, dyo = (int)((tap / 3) % 3) - 1, dxo = (int)(tap % 3) - 1;
        for (int i = 0; i < Cin; ++i)
            for (int o = 0; o < Cout; ++o) {
                double acc = 0.0;
                for (long z = 0; z < D; ++z)
                    for (long yy = 0; yy < H; ++yy)
                        for (long xx = 0; xx < W; ++xx) {
                            const long zz = orc_wrap(z + dz, D), y2 = orc_wrap(yy + dyo, H), x2 = orc_wrap(xx + dxo, W);
                            acc += x[((zz * H + y2) * W + x2) * Cin + i] *
                                   dy[((z * H + yy) * W + xx) * Cout + o];
                        }
                dw[(tap * Cin + i) * Cout + o] = acc;
            }
    }
    if (db)
        for (int o = 0; o < Cout; ++o) {
            double acc = 0.0;
            for (long c = 0; c < (long)D * H * W; ++c) acc += dy[c * Cout + o];
            db[o] = acc;
        }
}
