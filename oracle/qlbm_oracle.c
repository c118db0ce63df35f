/*
 * Oracle for the matrix-valued quantum lattice Boltzmann method
 * (C. B. Mendl, "Matrix-valued Quantum Lattice Boltzmann Method", 2015).
 *
 * TEST INFRASTRUCTURE ONLY.  This is a plain, slow, double-precision
 * restatement of the scheme of Sec. 3, written from the paper's equations
 * so that the CUDA library can be checked against it.  Only the test suite,
 * the package smoke check and the benchmark's CPU-baseline leg may load it;
 * the library never calls it, and the two share no code, header, table or
 * constant generator.
 *
 * Representation.  Every population W_i(x,t) is kept literally as a complex
 * 2x2 matrix (Sec. 2: W takes values in the Hermitian 2x2 matrices M_2),
 * and every step of Sec. 3.3 is written out on those matrices in the order
 * the paper gives it: moments (Eq. DiscrAvr), local equilibrium (Eq. WeqAlgo)
 * with the appendix coefficients, BGK collision (Eq. CollisionStep), then
 * streaming (Eq. TransportStep) on a periodic lattice, with two buffers.
 *
 * Exchange format with callers (the C ABI's canonical layout, so results can
 * be compared element by element): four reals per population in Pauli form
 * (f, s_x, s_y, s_z), W = (f*1 + s_x sigma_x + s_y sigma_y + s_z sigma_z)/2,
 * laid out [direction][component][site] with site = x + nx*(y + ny*z).
 * Directions are e_i = xi*(i1,i2[,i3]), i_k in {-1,0,1}, enumerated with i1
 * varying fastest, then i2, then i3, D3Q19 dropping the 8 cube corners
 * (Sec. 3.1); the opposite of direction q is b-1-q.
 *
 * Parity pins (tests/test_oracle_*.py): the printed constants of
 * Eqs. QuadSolution2Dmu0/3Dmu0 and of the appendix, the quadrature's defining
 * moment conditions (Eqs. quadrature2D/3D) checked by independent numerical
 * integration, the equilibrium's moment identities (Sec. 3.2), exact
 * conservation (Eqs. GlobalDensity, GlobalVelocity, GlobalTotalEnergy), the
 * equilibrium fixed point, the homogeneous closed form of BGK relaxation,
 * pure streaming against a library roll, Hermiticity, SU(2) covariance
 * (Sec. 2.1), the scalar reduction for W proportional to the identity, and
 * the adjoint against central finite differences of the forward step.
 * The Fermi-Dirac parameter inversion (Prop. 1, Eqs. nFDstdOmega and
 * energyFDstdOmega) is pinned by round trips from known parameters and by
 * closed forms of F_k; see the notes at that section.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;
typedef struct { cplx m[2][2]; } mat2;

#define QMAX 19

/* ------------------------------------------------------------------------- */
/* Riemann zeta, by P. Borwein's algorithm ("An efficient algorithm for the   */
/* Riemann zeta function", 2000, Algorithm 2): an accelerated alternating     */
/* (Dirichlet eta) series.  Used for the constants of Sec. 3.1 and the        */
/* appendix, which are stated in terms of zeta(3), zeta(3/2), zeta(5/2) and  */
/* zeta(7/2).                                                                 */
/* ------------------------------------------------------------------------- */
double oracle_zeta(double s)
{
    const int n = 40;
    double d[41];
    /* d_k = n * sum_{i<=k} (n+i-1)! 4^i / ((n-i)! (2i)!), built from the
       ratio of successive terms. */
    double term = 1.0, acc = 0.0;
    for (int i = 0; i <= n; ++i) {
        if (i > 0)
            term *= 4.0 * (double)(n + i - 1) * (double)(n - i + 1) /
                    ((double)(2 * i) * (double)(2 * i - 1));
        acc += term;
        d[i] = acc;
    }
    double sum = 0.0;
    for (int k = 0; k < n; ++k) {
        double sgn = (k % 2 == 0) ? 1.0 : -1.0;
        sum += sgn * (d[k] - d[n]) / pow((double)(k + 1), s);
    }
    return -sum / (d[n] * (1.0 - pow(2.0, 1.0 - s)));
}

/* ------------------------------------------------------------------------- */
/* Lattice and constants (Sec. 3.1, Sec. 3.2 and the appendix)               */
/* ------------------------------------------------------------------------- */
typedef struct {
    int d, b;
    int idx[QMAX][3];     /* lattice direction i (integer), e_i = xi * i */
    double w[QMAX];       /* quadrature weights w_i */
    double a, xi, beta0;  /* weight parameter a, lattice constant xi */
    double alpha_fac;
    /* alpha_1 = A1_0 + A1_1 * (beta0 eps), alpha_2 = A2_0 + A2_1 * (beta0 eps) */
    double A1_0, A1_1, A2_0, A2_1;
    double alpha3, alpha4, alpha5;
} lattice;

static int setup_lattice(int d, double beta0, lattice *L)
{
    if (d != 2 && d != 3) return -1;
    if (!(beta0 > 0.0)) return -1;
    memset(L, 0, sizeof(*L));
    L->d = d;
    L->beta0 = beta0;
    const double pi = M_PI, ln2 = log(2.0), s2 = sqrt(2.0);
    if (d == 2) {
        /* Eq. QuadSolution2Dmu0 and the appendix (d = 2). */
        double z3 = oracle_zeta(3.0);
        L->a = pi * pi * pi * pi / (972.0 * z3 * ln2);
        L->xi = (3.0 / pi) * sqrt(3.0 * z3 / beta0);
        L->alpha_fac = 72.0 * ln2 / (216.0 * ln2 * z3 - pi * pi * pi * pi);
        L->A1_0 = L->alpha_fac * 3.0 * z3;
        L->A1_1 = -L->alpha_fac * pi * pi / 6.0;
        L->A2_0 = -L->alpha_fac * pi * pi / 6.0;
        L->A2_1 = L->alpha_fac * 2.0 * ln2;
        L->alpha3 = 12.0 * ln2 / (pi * pi);
        L->alpha4 = L->alpha_fac * ln2;
        L->alpha5 = -L->alpha_fac * pi * pi / 6.0;
    } else {
        /* Eq. QuadSolution3Dmu0 and the appendix (d = 3). */
        double z32 = oracle_zeta(1.5), z52 = oracle_zeta(2.5), z72 = oracle_zeta(3.5);
        L->a = (41.0 + 9.0 * s2) * z52 * z52 / (558.0 * z32 * z72);
        L->xi = sqrt((3.0 / beta0) * (15.0 + 2.0 * s2) * z72 / (14.0 * z52));
        L->alpha_fac = 4.0 * z32 / (5.0 * (9.0 - 5.0 * s2) * z32 * z72 -
                                    3.0 * (9.0 - 4.0 * s2) * z52 * z52);
        L->A1_0 = L->alpha_fac * 1.25 * (9.0 - 5.0 * s2) * z72;
        L->A1_1 = -L->alpha_fac * (5.0 - 3.0 * s2) * z52;
        L->A2_0 = -L->alpha_fac * (5.0 - 3.0 * s2) * z52;
        L->A2_1 = L->alpha_fac * (6.0 - 4.0 * s2) * z32 * (2.0 / 3.0);
        L->alpha3 = 2.0 * z32 / ((3.0 + s2) * z52);
        L->alpha4 = L->alpha_fac * (3.0 - 2.0 * s2) * z32;
        L->alpha5 = -L->alpha_fac * (5.0 - 3.0 * s2) * z52;
    }
    /* Velocities and weights: D2Q9 w00 = 1-5a, w01 = a, w11 = a/4;
       D3Q19 w000 = 1-12a, w001 = a, w011 = a/2 (Eqs. QuadSolution2D/3D). */
    int q = 0;
    int kmin = (d == 3) ? -1 : 0, kmax = (d == 3) ? 1 : 0;
    for (int i3 = kmin; i3 <= kmax; ++i3)
        for (int i2 = -1; i2 <= 1; ++i2)
            for (int i1 = -1; i1 <= 1; ++i1) {
                int l1 = abs(i1) + abs(i2) + abs(i3);
                if (d == 3 && l1 == 3) continue;
                L->idx[q][0] = i1;
                L->idx[q][1] = i2;
                L->idx[q][2] = i3;
                if (l1 == 0) L->w[q] = (d == 2) ? 1.0 - 5.0 * L->a : 1.0 - 12.0 * L->a;
                else if (l1 == 1) L->w[q] = L->a;
                else L->w[q] = (d == 2) ? L->a / 4.0 : L->a / 2.0;
                ++q;
            }
    L->b = q;
    return 0;
}

/* Constants exported for the tests: a, xi, alpha_fac, A1_0, A1_1, A2_0, A2_1,
   alpha3, alpha4, alpha5, then b, then w[b], then idx[b][3]. */
int oracle_constants(int d, double beta0, double *out)
{
    lattice L;
    if (setup_lattice(d, beta0, &L)) return -1;
    int k = 0;
    out[k++] = L.a; out[k++] = L.xi; out[k++] = L.alpha_fac;
    out[k++] = L.A1_0; out[k++] = L.A1_1; out[k++] = L.A2_0; out[k++] = L.A2_1;
    out[k++] = L.alpha3; out[k++] = L.alpha4; out[k++] = L.alpha5;
    out[k++] = L.b;
    for (int q = 0; q < L.b; ++q) out[k++] = L.w[q];
    for (int q = 0; q < L.b; ++q)
        for (int j = 0; j < 3; ++j) out[k++] = L.idx[q][j];
    return k;
}

/* ------------------------------------------------------------------------- */
/* 2x2 complex helpers                                                        */
/* ------------------------------------------------------------------------- */
static inline double tr2(const mat2 *A) { return creal(A->m[0][0] + A->m[1][1]); }

static inline void mat_zero(mat2 *A) { memset(A, 0, sizeof(*A)); }

static inline void mat_axpy(mat2 *Y, double a, const mat2 *X)
{
    for (int j = 0; j < 2; ++j)
        for (int k = 0; k < 2; ++k) Y->m[j][k] += a * X->m[j][k];
}

/* Pauli form (f, s) <-> matrix W = (f 1 + s . sigma)/2. */
static inline void pauli_to_mat(double f, double sx, double sy, double sz, mat2 *W)
{
    W->m[0][0] = 0.5 * (f + sz);
    W->m[1][1] = 0.5 * (f - sz);
    W->m[0][1] = 0.5 * (sx - I * sy);
    W->m[1][0] = 0.5 * (sx + I * sy);
}

static inline void mat_to_pauli(const mat2 *W, double *f, double *sx, double *sy, double *sz)
{
    /* f = tr W, s_k = tr(W sigma_k). */
    *f = creal(W->m[0][0] + W->m[1][1]);
    *sx = creal(W->m[0][1] + W->m[1][0]);
    *sy = creal(I * (W->m[0][1] - W->m[1][0]));
    *sz = creal(W->m[0][0] - W->m[1][1]);
}

/* ------------------------------------------------------------------------- */
/* One site: moments, equilibrium, collision (Sec. 3.3)                       */
/* ------------------------------------------------------------------------- */
typedef struct {
    mat2 rho;
    double n;       /* tr rho */
    double u[3];
    double eps;
} moments;

/* Eq. DiscrAvr, written out literally:
     rho = sum_i W_i,
     tr[rho] u = sum_i e_i tr[W_i],
     tr[rho] eps = sum_i 1/2 |e_i - u|^2 tr[W_i]. */
static void site_moments(const lattice *L, const mat2 *W, moments *M)
{
    mat_zero(&M->rho);
    for (int i = 0; i < L->b; ++i) mat_axpy(&M->rho, 1.0, &W[i]);
    M->n = tr2(&M->rho);
    for (int k = 0; k < 3; ++k) {
        double acc = 0.0;
        for (int i = 0; i < L->b; ++i) acc += L->xi * L->idx[i][k] * tr2(&W[i]);
        M->u[k] = (k < L->d) ? acc / M->n : 0.0;
    }
    double acc = 0.0;
    for (int i = 0; i < L->b; ++i) {
        double d2 = 0.0;
        for (int k = 0; k < L->d; ++k) {
            double c = L->xi * L->idx[i][k] - M->u[k];
            d2 += c * c;
        }
        acc += 0.5 * d2 * tr2(&W[i]);
    }
    M->eps = acc / M->n;
}

/* The scalar factor of Eq. WeqAlgo:
     P_i = alpha1 + alpha2 beta0 |e_i|^2/2 + alpha3 beta0 (e_i.u)
           + alpha4 (beta0 e_i.u)^2 + alpha5 beta0 |u|^2/2,
   with alpha1, alpha2 from the appendix at eps_FD = eps. */
static double poly_P(const lattice *L, int i, const double *u, double eps)
{
    double b0 = L->beta0;
    double alpha1 = L->A1_0 + L->A1_1 * b0 * eps;
    double alpha2 = L->A2_0 + L->A2_1 * b0 * eps;
    double e2 = 0.0, eu = 0.0, u2 = 0.0;
    for (int k = 0; k < L->d; ++k) {
        double e = L->xi * L->idx[i][k];
        e2 += e * e;
        eu += e * u[k];
        u2 += u[k] * u[k];
    }
    return alpha1 + alpha2 * b0 * 0.5 * e2 + L->alpha3 * b0 * eu +
           L->alpha4 * (b0 * eu) * (b0 * eu) + L->alpha5 * b0 * 0.5 * u2;
}

/* Eq. WeqAlgo: W_i^eq = w_i rho P_i. */
static void site_equilibrium(const lattice *L, const moments *M, mat2 *Weq)
{
    for (int i = 0; i < L->b; ++i) {
        mat_zero(&Weq[i]);
        mat_axpy(&Weq[i], L->w[i] * poly_P(L, i, M->u, M->eps), &M->rho);
    }
}

/* Eq. CollisionStep: W_i^coll = W_i + (dt/tau)(W_i^eq - W_i). */
static void site_collide(const lattice *L, double omega, const mat2 *W, mat2 *Wc)
{
    moments M;
    mat2 Weq[QMAX];
    site_moments(L, W, &M);
    site_equilibrium(L, &M, Weq);
    for (int i = 0; i < L->b; ++i) {
        for (int j = 0; j < 2; ++j)
            for (int k = 0; k < 2; ++k)
                Wc[i].m[j][k] = W[i].m[j][k] + omega * (Weq[i].m[j][k] - W[i].m[j][k]);
    }
}

/* ------------------------------------------------------------------------- */
/* External magnetic field (Sec. 5, Eq. sigmaB_comm): the term                */
/* -i[mu sigma.B, W] added to the collision, integrated exactly over one     */
/* time step: W -> U W U*, U = exp(-i mu dt sigma.B)                          */
/*   = cos(phi) 1 - i sin(phi) (b.sigma), phi = mu dt |B|, b = B/|B|.          */
/* The field is one vector for the whole lattice (oracle_set_field) or one   */
/* per site, B(x) (oracle_set_field_array); U then depends on the site.      */
/* Off unless one of the two is set with mu |B| != 0.                         */
/* ------------------------------------------------------------------------- */
static double field_mu = 0.0, field_B[3] = {0.0, 0.0, 0.0};
static double *field_B_site = NULL;   /* [3][field_N], or NULL: uniform */
static int64_t field_N = 0;

void oracle_set_field(double mu, double Bx, double By, double Bz)
{
    free(field_B_site);
    field_B_site = NULL;
    field_N = 0;
    field_mu = mu;
    field_B[0] = Bx;
    field_B[1] = By;
    field_B[2] = Bz;
}

/* B [3][N]: B_x, B_y, B_z of every site; NULL switches the field off. */
int oracle_set_field_array(double mu, const double *B, int64_t N)
{
    free(field_B_site);
    field_B_site = NULL;
    field_N = 0;
    field_mu = 0.0;
    field_B[0] = field_B[1] = field_B[2] = 0.0;
    if (!B || N <= 0) return 0;
    field_B_site = (double *)malloc(3 * (size_t)N * sizeof(double));
    if (!field_B_site) return -2;
    memcpy(field_B_site, B, 3 * (size_t)N * sizeof(double));
    field_N = N;
    field_mu = mu;
    return 0;
}

/* The per-site field must cover the lattice it is used on. */
static int field_fits(int64_t N) { return field_B_site == NULL || field_N == N; }

/* U at site s of an N-site lattice; returns 0 (and leaves U) where the
   field vanishes. */
static int field_unitary(double dt, int64_t s, int64_t N, mat2 *U)
{
    double B[3];
    for (int k = 0; k < 3; ++k) B[k] = field_B_site ? field_B_site[(int64_t)k * N + s] : field_B[k];
    double nb = sqrt(B[0] * B[0] + B[1] * B[1] + B[2] * B[2]);
    if (!(nb > 0.0) || field_mu == 0.0) return 0;
    double phi = field_mu * dt * nb, c = cos(phi), sn = sin(phi);
    double bx = B[0] / nb, by = B[1] / nb, bz = B[2] / nb;
    /* b.sigma = [[bz, bx - i by], [bx + i by, -bz]] */
    U->m[0][0] = c - I * sn * bz;
    U->m[0][1] = -I * sn * (bx - I * by);
    U->m[1][0] = -I * sn * (bx + I * by);
    U->m[1][1] = c + I * sn * bz;
    return 1;
}

/* A -> X A Y for 2x2 complex matrices */
static void mat_sandwich(const mat2 *X, mat2 *A, const mat2 *Y)
{
    mat2 T, R;
    for (int j = 0; j < 2; ++j)
        for (int k = 0; k < 2; ++k) T.m[j][k] = X->m[j][0] * A->m[0][k] + X->m[j][1] * A->m[1][k];
    for (int j = 0; j < 2; ++j)
        for (int k = 0; k < 2; ++k) R.m[j][k] = T.m[j][0] * Y->m[0][k] + T.m[j][1] * Y->m[1][k];
    *A = R;
}

static void mat_adjoint(const mat2 *A, mat2 *B)
{
    for (int j = 0; j < 2; ++j)
        for (int k = 0; k < 2; ++k) B->m[j][k] = conj(A->m[k][j]);
}

/* ------------------------------------------------------------------------- */
/* Lattice helpers                                                            */
/* ------------------------------------------------------------------------- */
typedef struct { int64_t nx, ny, nz, N; } grid;

static int setup_grid(int d, const int64_t *dims, grid *G)
{
    G->nx = dims[0];
    G->ny = dims[1];
    G->nz = (d == 3) ? dims[2] : 1;
    if (G->nx <= 0 || G->ny <= 0 || G->nz <= 0) return -1;
    G->N = G->nx * G->ny * G->nz;
    return 0;
}

static inline int64_t wrap(int64_t a, int64_t n) { return ((a % n) + n) % n; }

/* Site reached from `site` by the integer displacement (dx,dy,dz), periodic. */
static inline int64_t shift_site(const grid *G, int64_t site, int dx, int dy, int dz)
{
    int64_t x = site % G->nx;
    int64_t y = (site / G->nx) % G->ny;
    int64_t z = site / (G->nx * G->ny);
    x = wrap(x + dx, G->nx);
    y = wrap(y + dy, G->ny);
    z = wrap(z + dz, G->nz);
    return x + G->nx * (y + G->ny * z);
}

static void state_from_pauli(const lattice *L, const grid *G, const double *p, mat2 *W)
{
    int64_t N = G->N;
    for (int64_t s = 0; s < N; ++s)
        for (int i = 0; i < L->b; ++i) {
            const double *c = p + (int64_t)i * 4 * N + s;
            pauli_to_mat(c[0], c[N], c[2 * N], c[3 * N], &W[s * L->b + i]);
        }
}

static void state_to_pauli(const lattice *L, const grid *G, const mat2 *W, double *p)
{
    int64_t N = G->N;
    for (int64_t s = 0; s < N; ++s)
        for (int i = 0; i < L->b; ++i) {
            double *c = p + (int64_t)i * 4 * N + s;
            mat_to_pauli(&W[s * L->b + i], &c[0], &c[N], &c[2 * N], &c[3 * N]);
        }
}

static int set_threads(int nthreads)
{
#ifdef _OPENMP
    omp_set_num_threads(nthreads > 0 ? nthreads : omp_get_num_procs());
    return omp_get_max_threads();
#else
    (void)nthreads;
    return 1;
#endif
}

int oracle_max_threads(int nthreads) { return set_threads(nthreads); }

/* ------------------------------------------------------------------------- */
/* Time stepping                                                              */
/* ------------------------------------------------------------------------- */
/* One full step t -> t + dt on matrix states: collision at every cell
   (Eq. CollisionStep), then W_i(x + dt e_i, t + dt) = W_i^coll(x, t)
   (Eq. TransportStep) with dt xi = dx, i.e. one cell along i, periodic. */
static void step_matrix(const lattice *L, const grid *G, double omega, double dt,
                        const mat2 *src, mat2 *dst)
{
    int64_t N = G->N;
    int b = L->b;
#pragma omp parallel for schedule(static)
    for (int64_t s = 0; s < N; ++s) {
        mat2 Wc[QMAX], U, Ud;
        site_collide(L, omega, &src[s * b], Wc);
        if (field_unitary(dt, s, N, &U)) {
            mat_adjoint(&U, &Ud);
            for (int i = 0; i < b; ++i) mat_sandwich(&U, &Wc[i], &Ud);   /* W -> U(x) W U(x)* */
        }
        for (int i = 0; i < b; ++i) {
            int64_t t = shift_site(G, s, L->idx[i][0], L->idx[i][1], L->idx[i][2]);
            dst[t * b + i] = Wc[i];
        }
    }
}

/* Runs nsteps on a state given as complex matrices, interleaved doubles
   [site][direction][row][col][re,im]. */
int oracle_run_matrix(int d, const int64_t *dims, double tau, double beta0, double dt,
                      int64_t nsteps, double *state_c, int nthreads)
{
    lattice L;
    grid G;
    if (setup_lattice(d, beta0, &L) || setup_grid(d, dims, &G)) return -1;
    if (!(tau > 0.0) || !(dt >= 0.0) || nsteps < 0 || !field_fits(G.N)) return -1;
    set_threads(nthreads);
    double omega = dt / tau;
    size_t bytes = (size_t)G.N * L.b * sizeof(mat2);
    mat2 *a = (mat2 *)state_c;
    mat2 *tmp = (mat2 *)malloc(bytes);
    if (!tmp) return -2;
    mat2 *src = a, *dst = tmp;
    for (int64_t n = 0; n < nsteps; ++n) {
        step_matrix(&L, &G, omega, dt, src, dst);
        mat2 *t = src; src = dst; dst = t;
    }
    if (src != a) memcpy(a, src, bytes);
    free(tmp);
    return 0;
}

/* Runs nsteps on a canonical Pauli state [b][4][N] in place. */
int oracle_run(int d, const int64_t *dims, double tau, double beta0, double dt,
               int64_t nsteps, double *state, int nthreads)
{
    lattice L;
    grid G;
    if (setup_lattice(d, beta0, &L) || setup_grid(d, dims, &G)) return -1;
    mat2 *W = (mat2 *)malloc((size_t)G.N * L.b * sizeof(mat2));
    if (!W) return -2;
    state_from_pauli(&L, &G, state, W);
    int rc = oracle_run_matrix(d, dims, tau, beta0, dt, nsteps, (double *)W, nthreads);
    if (rc == 0) state_to_pauli(&L, &G, W, state);
    free(W);
    return rc;
}

/* Collision of one site's populations (Pauli form [b][4]); no streaming.
   Used to evaluate single outputs of a full-size step one by one. */
int oracle_collide_site(int d, double tau, double beta0, double dt,
                        const double *pin, double *pout)
{
    lattice L;
    if (setup_lattice(d, beta0, &L)) return -1;
    mat2 W[QMAX], Wc[QMAX];
    memset(W, 0, sizeof(W));
    for (int i = 0; i < L.b; ++i)
        pauli_to_mat(pin[4 * i], pin[4 * i + 1], pin[4 * i + 2], pin[4 * i + 3], &W[i]);
    site_collide(&L, dt / tau, W, Wc);
    for (int i = 0; i < L.b; ++i)
        mat_to_pauli(&Wc[i], &pout[4 * i], &pout[4 * i + 1], &pout[4 * i + 2], &pout[4 * i + 3]);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Initial state, moments and global conserved quantities                     */
/* ------------------------------------------------------------------------- */
/* Equilibrium of one site from (rho, u, eps) given as Pauli density
   (n, S) with rho = (n 1 + S.sigma)/2 (Eq. WeqAlgo).  out is [b][4]. */
int oracle_equilibrium_site(int d, double beta0, const double *rho4, const double *u,
                            double eps, double *out)
{
    lattice L;
    if (setup_lattice(d, beta0, &L)) return -1;
    moments M;
    pauli_to_mat(rho4[0], rho4[1], rho4[2], rho4[3], &M.rho);
    M.n = rho4[0];
    for (int k = 0; k < 3; ++k) M.u[k] = (k < d) ? u[k] : 0.0;
    M.eps = eps;
    mat2 Weq[QMAX];
    site_equilibrium(&L, &M, Weq);
    for (int i = 0; i < L.b; ++i)
        mat_to_pauli(&Weq[i], &out[4 * i], &out[4 * i + 1], &out[4 * i + 2], &out[4 * i + 3]);
    return 0;
}

/* eps0: internal energy of the Fermi-Dirac distribution at the rule's own
   (beta0, mu0 = 0), Eq. energyFDstdOmega:
     eps0 = (d/2) beta0^-1 F_{d/2}(0) / F_{d/2-1}(0),
   with F_k(0) = -Li_{k+1}(-1) = (1 - 2^-k) zeta(k+1) for k > 0 and
   F_0(0) = log 2 (Sec. 2.2). */
double oracle_eps0(int d, double beta0)
{
    if (!(beta0 > 0.0)) return NAN;
    if (d == 2) return (0.5 * oracle_zeta(2.0)) / (log(2.0) * beta0);
    if (d == 3)
        return 1.5 * (1.0 - pow(2.0, -1.5)) * oracle_zeta(2.5) /
               ((1.0 - pow(2.0, -0.5)) * oracle_zeta(1.5) * beta0);
    return NAN;
}

/* Equilibrium initial state W_i(x, t0) = W_i^eq(rho(x), u(x), eps(x)).
   rho4 [4][N] (n, S_x, S_y, S_z), u [d][N], eps [N] or NULL (eps0). */
int oracle_init_equilibrium(int d, const int64_t *dims, double beta0, const double *rho4,
                            const double *u, const double *eps, double *state)
{
    lattice L;
    grid G;
    if (setup_lattice(d, beta0, &L) || setup_grid(d, dims, &G)) return -1;
    int64_t N = G.N;
    double eps0 = oracle_eps0(d, beta0);
    for (int64_t s = 0; s < N; ++s) {
        double r[4] = {rho4[s], rho4[N + s], rho4[2 * N + s], rho4[3 * N + s]};
        double uu[3] = {0, 0, 0};
        for (int k = 0; k < d; ++k) uu[k] = u[k * N + s];
        double e = eps ? eps[s] : eps0;
        double out[4 * QMAX];
        oracle_equilibrium_site(d, beta0, r, uu, e, out);
        for (int i = 0; i < L.b; ++i)
            for (int c = 0; c < 4; ++c) state[((int64_t)i * 4 + c) * N + s] = out[4 * i + c];
    }
    return 0;
}

/* Local moments of Eq. DiscrAvr at every site: rho4 [4][N] = (tr rho,
   tr(rho sigma_x), tr(rho sigma_y), tr(rho sigma_z)), u [d][N], eps [N]. */
int oracle_moments(int d, const int64_t *dims, double beta0, const double *state,
                   double *rho4, double *u, double *eps)
{
    lattice L;
    grid G;
    if (setup_lattice(d, beta0, &L) || setup_grid(d, dims, &G)) return -1;
    int64_t N = G.N;
    for (int64_t s = 0; s < N; ++s) {
        mat2 W[QMAX];
        for (int i = 0; i < L.b; ++i) {
            const double *c = state + (int64_t)i * 4 * N + s;
            pauli_to_mat(c[0], c[N], c[2 * N], c[3 * N], &W[i]);
        }
        moments M;
        site_moments(&L, W, &M);
        mat_to_pauli(&M.rho, &rho4[s], &rho4[N + s], &rho4[2 * N + s], &rho4[3 * N + s]);
        for (int k = 0; k < d; ++k) u[k * N + s] = M.u[k];
        eps[s] = M.eps;
    }
    return 0;
}

/* Global averages of Eqs. GlobalDensity, GlobalVelocity, GlobalTotalEnergy:
   out[0..3] = Pauli components of (1/|Lambda|) sum_x rho(x),
   out[4..6] = (1/|Lambda|) sum_x sum_i e_i tr W_i (zero beyond d),
   out[7]    = (1/|Lambda|) sum_x sum_i |e_i|^2/2 tr W_i. */
int oracle_conserved(int d, const int64_t *dims, double beta0, const double *state,
                     double *out)
{
    lattice L;
    grid G;
    if (setup_lattice(d, beta0, &L) || setup_grid(d, dims, &G)) return -1;
    int64_t N = G.N;
    mat2 rho;
    mat_zero(&rho);
    double mom[3] = {0, 0, 0}, en = 0.0;
    for (int64_t s = 0; s < N; ++s)
        for (int i = 0; i < L.b; ++i) {
            const double *c = state + (int64_t)i * 4 * N + s;
            mat2 W;
            pauli_to_mat(c[0], c[N], c[2 * N], c[3 * N], &W);
            mat_axpy(&rho, 1.0, &W);
            double t = tr2(&W), e2 = 0.0;
            for (int k = 0; k < d; ++k) {
                double e = L.xi * L.idx[i][k];
                mom[k] += e * t;
                e2 += e * e;
            }
            en += 0.5 * e2 * t;
        }
    double inv = 1.0 / (double)N;
    mat_to_pauli(&rho, &out[0], &out[1], &out[2], &out[3]);
    for (int k = 0; k < 4; ++k) out[k] *= inv;
    for (int k = 0; k < 3; ++k) out[4 + k] = mom[k] * inv;
    out[7] = en * inv;
    return 0;
}

/* Smallest eigenvalue of every discrete equilibrium W_i^eq = w_i rho P_i
   (Eq. WeqAlgo) formed from the moments of the given state, i.e. of the
   equilibria the next collision relaxes towards.  Sec. 3.2 (end) and
   Sec. 3.3 (end) note that these can have negative eigenvalues and that the
   scheme does not clip them; this diagnostic exposes where.  Literally: for
   the Hermitian 2x2 matrix [[a, c], [conj(c), e]] the eigenvalues are
   (a + e)/2 -+ sqrt(((a - e)/2)^2 + |c|^2).  out [b][N]. */
int oracle_eq_min_eigenvalues(int d, const int64_t *dims, double beta0, const double *state, double *out)
{
    lattice L;
    grid G;
    if (setup_lattice(d, beta0, &L) || setup_grid(d, dims, &G)) return -1;
    int64_t N = G.N;
    for (int64_t s = 0; s < N; ++s) {
        mat2 W[QMAX], Weq[QMAX];
        for (int i = 0; i < L.b; ++i) {
            const double *c = state + (int64_t)i * 4 * N + s;
            pauli_to_mat(c[0], c[N], c[2 * N], c[3 * N], &W[i]);
        }
        moments M;
        site_moments(&L, W, &M);
        site_equilibrium(&L, &M, Weq);
        for (int i = 0; i < L.b; ++i) {
            double a = creal(Weq[i].m[0][0]), e = creal(Weq[i].m[1][1]);
            double off = cabs(Weq[i].m[0][1]);
            double half = 0.5 * (a - e);
            out[(int64_t)i * N + s] = 0.5 * (a + e) - sqrt(half * half + off * off);
        }
    }
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Adjoint (discrete, reverse mode) of one step                               */
/* ------------------------------------------------------------------------- */
/* Cotangents are Hermitian matrices L with dJ = sum tr(L dW); in the Pauli
   exchange format a cotangent (l_f, l_s) stands for L = l_f 1 + l_s.sigma,
   i.e. l_f = dJ/df and l_s = dJ/ds for W = (f 1 + s.sigma)/2.
   Reverse of the forward order: streaming is a permutation, so its adjoint
   pulls L'_i(x) = L^{n+1}_i(x + e_i); then the collision's chain rule
   through W^eq = w_i rho P_i(u, eps), eps and u (Eq. DiscrAvr) back to W. */
static void site_collide_adjoint(const lattice *L, double omega, double dom_dtau,
                                 const mat2 *W, const mat2 *Lp, mat2 *Lout,
                                 double *dJ_dtau)
{
    int b = L->b, d = L->d;
    double b0 = L->beta0;
    moments M;
    mat2 Weq[QMAX];
    site_moments(L, W, &M);
    site_equilibrium(L, &M, Weq);

    /* dJ/dtau through omega = dt/tau: sum_i tr(L'_i (W_i^eq - W_i)) domega/dtau. */
    double acc = 0.0;
    for (int i = 0; i < b; ++i)
        for (int j = 0; j < 2; ++j)
            for (int k = 0; k < 2; ++k)
                acc += creal(Lp[i].m[k][j] * (Weq[i].m[j][k] - W[i].m[j][k]));
    *dJ_dtau += acc * dom_dtau;

    /* W_i' = (1-omega) W_i + omega W_i^eq. */
    mat2 rhobar;
    mat_zero(&rhobar);
    double ubar[3] = {0, 0, 0}, epsbar = 0.0;
    double alpha1p = L->A1_1 * b0, alpha2p = L->A2_1 * b0; /* d alpha / d eps */
    for (int i = 0; i < b; ++i) {
        Lout[i] = Lp[i];
        for (int j = 0; j < 2; ++j)
            for (int k = 0; k < 2; ++k) Lout[i].m[j][k] *= (1.0 - omega);
        double P = poly_P(L, i, M.u, M.eps);
        /* W_i^eq = w_i P_i rho: rho gets w_i P_i omega L'_i, P_i gets
           w_i omega tr(L'_i rho). */
        mat_axpy(&rhobar, omega * L->w[i] * P, &Lp[i]);
        double Pbar = 0.0;
        for (int j = 0; j < 2; ++j)
            for (int k = 0; k < 2; ++k) Pbar += creal(Lp[i].m[k][j] * M.rho.m[j][k]);
        Pbar *= omega * L->w[i];
        double e[3] = {0, 0, 0}, e2 = 0.0, eu = 0.0;
        for (int k = 0; k < d; ++k) {
            e[k] = L->xi * L->idx[i][k];
            e2 += e[k] * e[k];
            eu += e[k] * M.u[k];
        }
        /* dP/du = alpha3 beta0 e + 2 alpha4 beta0^2 (e.u) e + alpha5 beta0 u,
           dP/deps = alpha1' + alpha2' beta0 |e|^2/2. */
        for (int k = 0; k < d; ++k)
            ubar[k] += Pbar * (L->alpha3 * b0 * e[k] + 2.0 * L->alpha4 * b0 * b0 * eu * e[k] +
                               L->alpha5 * b0 * M.u[k]);
        epsbar += Pbar * (alpha1p + alpha2p * b0 * 0.5 * e2);
    }
    /* eps = (1/n) sum_j |e_j - u|^2/2 tr W_j: d eps/d tr W_j =
       (|e_j - u|^2/2 - eps)/n; d eps/du = -(1/n) sum_j (e_j - u) tr W_j = 0.
       u = (1/n) sum_j e_j tr W_j: d u/d tr W_j = (e_j - u)/n.
       rho = sum_j W_j. */
    for (int j = 0; j < b; ++j) {
        double e[3] = {0, 0, 0}, d2 = 0.0, du = 0.0;
        for (int k = 0; k < d; ++k) {
            e[k] = L->xi * L->idx[j][k];
            d2 += (e[k] - M.u[k]) * (e[k] - M.u[k]);
            du += ubar[k] * (e[k] - M.u[k]);
        }
        double tbar = epsbar * (0.5 * d2 - M.eps) / M.n + du / M.n;
        mat_axpy(&Lout[j], 1.0, &rhobar);
        Lout[j].m[0][0] += tbar;
        Lout[j].m[1][1] += tbar;
    }
}

/* One adjoint step: given the state W^n (Pauli [b][4][N]) and the cotangent
   of W^{n+1} (Pauli-cotangent [b][4][N]), returns the cotangent of W^n and
   adds the step's contribution to dJ/dtau. */
int oracle_adjoint_step(int d, const int64_t *dims, double tau, double beta0, double dt,
                        const double *state, const double *lam_next, double *lam,
                        double *dJ_dtau, int nthreads)
{
    lattice L;
    grid G;
    if (setup_lattice(d, beta0, &L) || setup_grid(d, dims, &G)) return -1;
    set_threads(nthreads);
    int64_t N = G.N;
    int b = L.b;
    double omega = dt / tau, dom_dtau = -dt / (tau * tau);
    double total = 0.0;
    if (!field_fits(N)) return -1;
#pragma omp parallel for schedule(static) reduction(+ : total)
    for (int64_t s = 0; s < N; ++s) {
        mat2 W[QMAX], Lp[QMAX], Lo[QMAX], U, Ud;
        int field = field_unitary(dt, s, N, &U);
        if (field) mat_adjoint(&U, &Ud);
        for (int i = 0; i < b; ++i) {
            const double *c = state + (int64_t)i * 4 * N + s;
            pauli_to_mat(c[0], c[N], c[2 * N], c[3 * N], &W[i]);
            int64_t t = shift_site(&G, s, L.idx[i][0], L.idx[i][1], L.idx[i][2]);
            const double *l = lam_next + (int64_t)i * 4 * N + t;
            /* cotangent matrix L = l_f 1 + l_s . sigma */
            Lp[i].m[0][0] = l[0] + l[3 * N];
            Lp[i].m[1][1] = l[0] - l[3 * N];
            Lp[i].m[0][1] = l[N] - I * l[2 * N];
            Lp[i].m[1][0] = l[N] + I * l[2 * N];
            /* W_rot = U W_c U*: dJ = tr(L' U dW_c U*) = tr(U* L' U dW_c) */
            if (field) mat_sandwich(&Ud, &Lp[i], &U);
        }
        double part = 0.0;
        site_collide_adjoint(&L, omega, dom_dtau, W, Lp, Lo, &part);
        total += part;
        for (int i = 0; i < b; ++i) {
            double *o = lam + (int64_t)i * 4 * N + s;
            /* back to (l_f, l_s): l_f = tr L / 2, l_s = tr(L sigma) / 2 */
            o[0] = 0.5 * creal(Lo[i].m[0][0] + Lo[i].m[1][1]);
            o[N] = 0.5 * creal(Lo[i].m[0][1] + Lo[i].m[1][0]);
            o[2 * N] = 0.5 * creal(I * (Lo[i].m[0][1] - Lo[i].m[1][0]));
            o[3 * N] = 0.5 * creal(Lo[i].m[0][0] - Lo[i].m[1][1]);
        }
    }
    *dJ_dtau += total;
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Fermi-Dirac integrals and the parameters of a Fermi-Dirac equilibrium     */
/* (Sec. 2.2: Prop. 1, Eqs. nFDstdOmega and energyFDstdOmega).               */
/*                                                                           */
/* F_k(x) = Gamma(k+1)^-1 int_0^inf t^k / (e^(t-x) + 1) dt, written with      */
/* t = s^2 as 2/Gamma(k+1) int_0^inf s^(2k+1) / (e^(s^2-x) + 1) ds, whose     */
/* integrand is smooth for k >= -1/2, and integrated by adaptive composite   */
/* 20-point Gauss-Legendre quadrature (nodes from Newton's method on the     */
/* Legendre recurrence), split at the Fermi edge s = sqrt(x).  F_0 and       */
/* F_-1 use the closed forms the paper states.                               */
/* ------------------------------------------------------------------------- */
#define GLN 20
static double gl_x[GLN], gl_w[GLN];
static int gl_ready = 0;

static void gl_setup(void)
{
    if (gl_ready) return;
    for (int i = 0; i < GLN; ++i) {
        double z = cos(M_PI * (i + 0.75) / (GLN + 0.5)), pp = 0.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;   /* P_0, P_1 */
            for (int n = 2; n <= GLN; ++n) {
                double p2 = ((2.0 * n - 1.0) * z * p1 - (n - 1.0) * p0) / n;
                p0 = p1;
                p1 = p2;
            }
            pp = GLN * (z * p1 - p0) / (z * z - 1.0);   /* P_n' */
            double dz = p1 / pp;
            z -= dz;
            if (fabs(dz) < 1e-17) break;
        }
        gl_x[i] = z;
        gl_w[i] = 2.0 / ((1.0 - z * z) * pp * pp);
    }
    gl_ready = 1;
}

static double fermi(double a)   /* 1/(e^a + 1) without overflow */
{
    if (a > 0.0) {
        double e = exp(-a);
        return e / (1.0 + e);
    }
    return 1.0 / (1.0 + exp(a));
}

static double fd_integrand(double s, double k, double x)
{
    return 2.0 * pow(s, 2.0 * k + 1.0) * fermi(s * s - x);
}

static double gl_panel(double a, double b, double k, double x)
{
    double c = 0.5 * (a + b), h = 0.5 * (b - a), acc = 0.0;
    for (int i = 0; i < GLN; ++i) acc += gl_w[i] * fd_integrand(c + h * gl_x[i], k, x);
    return acc * h;
}

/* Bisects a panel until its two halves agree with the whole to within
   tol_abs (a fixed fraction of the whole integral, so panels where the
   integrand is negligible stop at once) or to rounding level. */
static double gl_adaptive(double a, double b, double k, double x, double whole, double tol_abs,
                          int depth)
{
    double m = 0.5 * (a + b);
    double l = gl_panel(a, m, k, x), r = gl_panel(m, b, k, x);
    double diff = fabs(l + r - whole);
    if (depth >= 30 || diff <= tol_abs || diff <= 8e-16 * (fabs(l) + fabs(r))) return l + r;
    return gl_adaptive(a, m, k, x, l, 0.5 * tol_abs, depth + 1) +
           gl_adaptive(m, b, k, x, r, 0.5 * tol_abs, depth + 1);
}

/* Complete Fermi-Dirac integral F_k(x), k = -1, 0 or a value >= -1/2. */
double oracle_fd(double k, double x)
{
    if (k == -1.0) return fermi(-x);                                   /* (1 + e^-x)^-1 */
    if (k == 0.0) return x > 0.0 ? x + log1p(exp(-x)) : log1p(exp(x)); /* log(1 + e^x) */
    if (k < -0.5) return NAN;
    gl_setup();
    double xe = x > 0.0 ? x : 0.0;
    double edge = sqrt(xe), top = sqrt(xe + 80.0);
    double p1 = edge > 0.0 ? gl_panel(0.0, edge, k, x) : 0.0;
    double p2 = gl_panel(edge, top, k, x);
    double tol = 1e-15 * (fabs(p1) + fabs(p2));
    double acc = 0.0;
    if (edge > 0.0) acc += gl_adaptive(0.0, edge, k, x, p1, tol, 0);
    acc += gl_adaptive(edge, top, k, x, p2, tol, 0);
    return acc / tgamma(k + 1.0);
}

/* Forward map (Eqs. nFDstdOmega, energyFDstdOmega): densities of the two
   spin species and the internal energy of the Fermi-Dirac distribution with
   parameters (beta, mu_up, mu_dn).  out = {n_up, n_dn, eps}. */
int oracle_fd_moments(int d, double beta, double mu_up, double mu_dn, double *out)
{
    if ((d != 2 && d != 3) || !(beta > 0.0)) return -1;
    double h = 0.5 * d, pre = pow(2.0 * M_PI / beta, h);
    double nu = pre * oracle_fd(h - 1.0, beta * mu_up);
    double nd = pre * oracle_fd(h - 1.0, beta * mu_dn);
    double e = h / beta * (oracle_fd(h, beta * mu_up) + oracle_fd(h, beta * mu_dn)) /
               (oracle_fd(h - 1.0, beta * mu_up) + oracle_fd(h - 1.0, beta * mu_dn));
    out[0] = nu;
    out[1] = nd;
    out[2] = e;
    return 0;
}

/* nu solving (2 pi / beta)^h F_{h-1}(nu) = n_s: closed form in 2D
   (F_0(nu) = log(1 + e^nu)); safeguarded Newton (derivative F_{h-2}) on a
   bisection bracket in 3D. */
static double species_nu(int d, double beta, double ns)
{
    double h = 0.5 * d, y = ns * pow(beta / (2.0 * M_PI), h);
    if (d == 2) return y > 30.0 ? y + log(-expm1(-y)) : log(expm1(y));
    double lo = log(y) - 10.0, hi = (y > 1.0 ? pow(y * tgamma(h + 1.0), 1.0 / h) : log(y)) + 10.0;
    double nu = 0.5 * (lo + hi);
    for (int it = 0; it < 200; ++it) {
        double F = oracle_fd(h - 1.0, nu) - y;
        if (F > 0.0) hi = nu;
        else lo = nu;
        double step = F / oracle_fd(h - 2.0, nu);
        double nn = nu - step;
        if (!(nn > lo && nn < hi)) nn = 0.5 * (lo + hi);
        if (fabs(nn - nu) <= 1e-15 * (1.0 + fabs(nu)) || hi - lo <= 1e-15 * (1.0 + fabs(nu))) {
            nu = nn;
            break;
        }
        nu = nn;
    }
    return nu;
}

/* Prop. 1 inverted: the parameters (beta, mu_up, mu_dn) and eigenbasis of the
   Fermi-Dirac equilibrium whose density matrix rho = (n 1 + S.sigma)/2 and
   internal energy eps are given.  The eigen-decomposition of rho is taken on
   the complex 2x2 matrix (characteristic polynomial, eigenvector of the larger
   eigenvalue), the Bloch axis is that eigenvector's <v|sigma|v>.  beta is
   found by bisection on log(beta) of
     g(beta) = (d/2) beta^-1 (2 pi/beta)^(d/2) sum_s F_{d/2}(nu_s(beta)) - n eps,
   decreasing in beta, bracketed around the classical estimate (d/2)/eps.
   out = {beta, mu_up, mu_dn, a_x, a_y, a_z}; returns 0, 1 if rho is not
   positive definite, 2 if no beta fits (eps below the degenerate limit). */
int oracle_fd_params(int d, const double *rho4, double eps, double *out)
{
    if (d != 2 && d != 3) return -1;
    for (int i = 0; i < 6; ++i) out[i] = NAN;
    mat2 r;
    pauli_to_mat(rho4[0], rho4[1], rho4[2], rho4[3], &r);
    double tr = creal(r.m[0][0] + r.m[1][1]);
    double det = creal(r.m[0][0] * r.m[1][1] - r.m[0][1] * r.m[1][0]);
    double disc = sqrt(fmax(0.25 * tr * tr - det, 0.0));
    double lup = 0.5 * tr + disc, ldn = 0.5 * tr - disc;
    if (!(ldn > 0.0)) return 1;
    /* eigenvector of lup: (r01, lup - r00) or (lup - r11, r10), the longer one */
    cplx v0 = r.m[0][1], v1 = lup - r.m[0][0];
    cplx w0 = lup - r.m[1][1], w1 = r.m[1][0];
    if (cabs(w0) * cabs(w0) + cabs(w1) * cabs(w1) > cabs(v0) * cabs(v0) + cabs(v1) * cabs(v1)) {
        v0 = w0;
        v1 = w1;
    }
    double nv = sqrt(creal(v0 * conj(v0) + v1 * conj(v1)));
    if (nv > 0.0 && disc > 0.0) {
        v0 /= nv;
        v1 /= nv;
        out[3] = 2.0 * creal(conj(v0) * v1);          /* <v|sigma_x|v> */
        out[4] = 2.0 * cimag(conj(v0) * v1);          /* <v|sigma_y|v> */
        out[5] = creal(conj(v0) * v0 - conj(v1) * v1); /* <v|sigma_z|v> */
    } else {
        out[3] = out[4] = out[5] = 0.0;               /* degenerate: any axis */
    }
    double h = 0.5 * d, nE = tr * eps;
    if (!(eps > 0.0)) return 2;
#define G_OF(lb)                                                                            \
    (h * exp(-(lb)) * pow(2.0 * M_PI * exp(-(lb)), h) *                                      \
         (oracle_fd(h, species_nu(d, exp(lb), lup)) + oracle_fd(h, species_nu(d, exp(lb), ldn))) - \
     nE)
    /* bracket around the classical estimate beta = (d/2)/eps, widened by e */
    double lb0 = log(h / eps), blo = lb0 - 1.0, bhi = lb0 + 1.0;
    int tries = 0;
    while (!(G_OF(blo) > 0.0)) {
        blo -= 1.0;
        if (++tries > 30) return 2;
    }
    tries = 0;
    while (!(G_OF(bhi) < 0.0)) {
        bhi += 1.0;
        if (++tries > 30) return 2;
    }
    for (int it = 0; it < 200 && bhi - blo > 1e-15 * (1.0 + fabs(blo)); ++it) {
        double mid = 0.5 * (blo + bhi), gm = G_OF(mid);
        if (gm > 0.0) blo = mid;
        else bhi = mid;
    }
#undef G_OF
    double beta = exp(0.5 * (blo + bhi));
    out[0] = beta;
    out[1] = species_nu(d, beta, lup) / beta;
    out[2] = species_nu(d, beta, ldn) / beta;
    return 0;
}
