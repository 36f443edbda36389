/*
 * Plain FP64 CPU oracle of the lattice Boltzmann hot path.
 *
 * TEST INFRASTRUCTURE ONLY. Only the tests, the smoke check and the benchmark's
 * CPU-baseline leg may load this code. It shares no source, header, table or
 * helper with the CUDA library: the velocity sets, the equilibrium, the collision
 * operators, the streaming and the adjoint are written out here on their own,
 * node by node, in the order the paper states them. It is deliberately slow.
 * Build: gcc -O2 -ffp-contract=off -fopenmp -shared -fPIC (no fused multiply-add).
 *
 * Passages followed (Bedrunka et al., "Lettuce", arXiv 2106.12929):
 *   Eq. 1  lattice Boltzmann equation f_i(x + c_i, t + 1) = f_i(x, t) + Omega_i(f)
 *          -> ora_step: collide each node, then push f*_i to x + c_i.
 *   Eq. 2  BGK collision Omega_i = -(f_i - f_i^eq)/tau.
 *   Eq. 3  second-order equilibrium.
 *   Eq. 4  density and momentum moments.
 *   Sec. 2.1 regularized collision (Latt & Chopard): rebuild f^neq from Pi^neq.
 *   Eq. 5  moment-space collision Omega = -M^-1 S^-1 (M f - m^eq) with
 *          conserved rates 1, shear tau_n = nu/c_s^2 + 1/2, higher-moment rates
 *          tau = exp(net) + 1/2 from a per-node network of local moments (Sec. 3.1).
 *   Sec. 2.1 further collision models the paper lists by citation only:
 *          two-relaxation-time (Ginzburg 2008), moment-space MRT with fixed rates
 *          (Eq. 5 with constant higher-moment relaxation times), and the entropic
 *          KBC model (Karlin, Boesch & Chikatamarla 2014). Their definitions are
 *          written out at collide_node.
 *          A second network follows the shape Sec. 3.1 describes: one hidden layer
 *          and three outputs, one relaxation time exp(z_n) + 1/2 per higher moment.
 *   Eq. 6  training loss from velocity, vorticity and energy mismatch.
 *   Sec. 3.2 gradients through the solver (here: the discrete adjoint, by hand), and
 *          the velocity-shift forcing of the spectral control: BGK toward
 *          f^eq(rho, u + du) -> ora_step_ushift (du itself is computed in spectral.py).
 *   Sec. 2.2 boundary conditions (listed without formulas): halfway bounce-back on
 *          solid nodes with the moving-wall term -> ora_step_walls.
 * Readings where the paper is silent (stencil order, Guo forcing, Hermite moment
 * basis, the six network inputs, loss normalisation) are stated at each function.
 *
 * Parity pins: every function here is checked by tests against closed forms,
 * invariants, brute force or finite differences (tests/test_oracle_*.py).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORA_OK 0
#define ORA_ERR_ARG 1
#define ORA_ERR_OOM 2

/* collision kinds (same numbering as the library's public enum, written here on its own) */
#define ORA_BGK 0
#define ORA_REG 1
#define ORA_LEARNED 2
#define ORA_NONE 3
#define ORA_TRT 4
#define ORA_KBC 5
#define ORA_MRT 6
#define ORA_LEARNED3 7

#define NH 24                 /* hidden width of the per-node network */
#define NIN 6                 /* number of network inputs (moment invariants) */
#define NTHETA (NH * NIN + NH + NH * NH + NH + NH + 1) /* 793 */
#define NMLP (NTHETA + 2 * NIN) /* parameters + input shift[6] + input scale[6] */
#define NH3 53                  /* hidden width of the one-hidden-layer, three-output network */
#define NTHETA3 (NH3 * NIN + NH3 + 3 * NH3 + 3) /* 533 */
#define NMLP3 (NTHETA3 + 2 * NIN)

typedef struct {
    int d, q;
    int c[27][3];
    double w[27];
    int opp[27];
} stencil_t;

static const double cs2 = 1.0 / 3.0;

/* ------------------------------------------------------------------------ */
/* Velocity sets. The paper names D2Q9, D3Q19 and D3Q27 (Sec. 2.2, 3.1, 3.3)  */
/* but prints no table. Order used: rest, then the +/- axis pairs, then the  */
/* edge pairs (xy, xz, yz families), then the corner pairs. Weights follow   */
/* from |c|^2 (textbook values, Krueger et al. 2016).                        */
/* ------------------------------------------------------------------------ */
static int stencil_get(int st, stencil_t* s)
{
    static const int d2q9[9][3] = {{0, 0, 0}, {1, 0, 0}, {-1, 0, 0}, {0, 1, 0}, {0, -1, 0},
                                   {1, 1, 0}, {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0}};
    static const int d3q27[27][3] = {
        {0, 0, 0},
        {1, 0, 0}, {-1, 0, 0}, {0, 1, 0}, {0, -1, 0}, {0, 0, 1}, {0, 0, -1},
        {1, 1, 0}, {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0},
        {1, 0, 1}, {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1},
        {0, 1, 1}, {0, -1, -1}, {0, 1, -1}, {0, -1, 1},
        {1, 1, 1}, {-1, -1, -1}, {1, 1, -1}, {-1, -1, 1},
        {1, -1, 1}, {-1, 1, -1}, {-1, 1, 1}, {1, -1, -1}};
    int i, j, a;
    memset(s, 0, sizeof(*s));
    if (st == 0) {
        s->d = 2; s->q = 9;
        for (i = 0; i < 9; ++i) for (a = 0; a < 3; ++a) s->c[i][a] = d2q9[i][a];
    } else if (st == 1 || st == 2) {
        s->d = 3; s->q = (st == 1) ? 19 : 27;
        for (i = 0; i < s->q; ++i) for (a = 0; a < 3; ++a) s->c[i][a] = d3q27[i][a];
    } else {
        return ORA_ERR_ARG;
    }
    for (i = 0; i < s->q; ++i) {
        int c2 = s->c[i][0] * s->c[i][0] + s->c[i][1] * s->c[i][1] + s->c[i][2] * s->c[i][2];
        if (st == 0) s->w[i] = (c2 == 0) ? 4.0 / 9.0 : (c2 == 1) ? 1.0 / 9.0 : 1.0 / 36.0;
        else if (st == 1) s->w[i] = (c2 == 0) ? 1.0 / 3.0 : (c2 == 1) ? 1.0 / 18.0 : 1.0 / 36.0;
        else s->w[i] = (c2 == 0) ? 8.0 / 27.0 : (c2 == 1) ? 2.0 / 27.0 : (c2 == 2) ? 1.0 / 54.0 : 1.0 / 216.0;
    }
    /* opposite directions found by search, not listed */
    for (i = 0; i < s->q; ++i) {
        s->opp[i] = -1;
        for (j = 0; j < s->q; ++j)
            if (s->c[j][0] == -s->c[i][0] && s->c[j][1] == -s->c[i][1] && s->c[j][2] == -s->c[i][2])
                s->opp[i] = j;
    }
    return ORA_OK;
}

int ora_stencil(int st, int* d, int* q, int* c, double* w, int* opp)
{
    stencil_t s;
    int i, a;
    if (stencil_get(st, &s)) return ORA_ERR_ARG;
    *d = s.d; *q = s.q;
    for (i = 0; i < s.q; ++i) {
        for (a = 0; a < 3; ++a) c[3 * i + a] = s.c[i][a];
        w[i] = s.w[i];
        opp[i] = s.opp[i];
    }
    return ORA_OK;
}

/* ------------------------------------------------------------------------ */
/* Grid helpers: node n = x + nx (y + ny z), periodic in every direction.    */
/* ------------------------------------------------------------------------ */
static int64_t wrap(int64_t v, int64_t n) { v %= n; return v < 0 ? v + n : v; }

static int64_t shifted_node(const int64_t* dims, int64_t n, int sx, int sy, int sz)
{
    int64_t nx = dims[0], ny = dims[1], nz = dims[2];
    int64_t x = n % nx, y = (n / nx) % ny, z = n / (nx * ny);
    return wrap(x + sx, nx) + nx * (wrap(y + sy, ny) + ny * wrap(z + sz, nz));
}

static int check_dims(const stencil_t* s, const int64_t* dims)
{
    if (dims[0] < 1 || dims[1] < 1 || dims[2] < 1) return ORA_ERR_ARG;
    if (s->d == 2 && dims[2] != 1) return ORA_ERR_ARG;
    return ORA_OK;
}

/* ------------------------------------------------------------------------ */
/* Eq. 3 equilibrium and Eq. 4 moments of one node.                          */
/* ------------------------------------------------------------------------ */
static void equilibrium(const stencil_t* s, double rho, const double* u, double* feq)
{
    int i;
    double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    for (i = 0; i < s->q; ++i) {
        double cu = s->c[i][0] * u[0] + s->c[i][1] * u[1] + s->c[i][2] * u[2];
        feq[i] = s->w[i] * rho * (1.0 + cu / cs2 + (cu * cu) / (2.0 * cs2 * cs2) - uu / (2.0 * cs2));
    }
}

/* rho = sum f, rho u = sum c f; with a body force the velocity carries the Guo
 * half-force shift u = (sum c f + F/2) / rho (reading: Guo, Zheng & Shi 2002). */
static void node_moments(const stencil_t* s, const double* f, const double* F, double* rho, double* u)
{
    int i, a;
    double r = 0.0, j[3] = {0.0, 0.0, 0.0};
    for (i = 0; i < s->q; ++i) {
        r += f[i];
        for (a = 0; a < 3; ++a) j[a] += s->c[i][a] * f[i];
    }
    for (a = 0; a < 3; ++a) u[a] = (j[a] + (F ? 0.5 * F[a] : 0.0)) / r;
    *rho = r;
}

/* Guo source term S_i = (1 - omega/2) w_i [ (c_i - u)/c_s^2 + (c_i.u) c_i / c_s^4 ] . F */
static void guo_source(const stencil_t* s, double omega, const double* u, const double* F, double* S)
{
    int i, a;
    for (i = 0; i < s->q; ++i) {
        double cu = s->c[i][0] * u[0] + s->c[i][1] * u[1] + s->c[i][2] * u[2];
        double acc = 0.0;
        for (a = 0; a < 3; ++a)
            acc += ((s->c[i][a] - u[a]) / cs2 + cu * s->c[i][a] / (cs2 * cs2)) * F[a];
        S[i] = (1.0 - 0.5 * omega) * s->w[i] * acc;
    }
}

int ora_guo_source(int st, double tau, const double* u, const double* F, double* S)
{
    stencil_t s;
    double uu[3] = {u[0], u[1], 0.0}, FF[3] = {F[0], F[1], 0.0};
    if (stencil_get(st, &s)) return ORA_ERR_ARG;
    if (s.d == 3) { uu[2] = u[2]; FF[2] = F[2]; }
    guo_source(&s, 1.0 / tau, uu, FF, S);
    return ORA_OK;
}

/* ------------------------------------------------------------------------ */
/* D2Q9 moment basis for the Eq. 5 collision. Dellar's matrix is not printed; */
/* the reading used is the Hermite basis with the same split into conserved, */
/* stress and higher (ghost) moments:                                        */
/*   1, cx, cy, cx^2-cs2, cx cy, cy^2-cs2, (cx^2-cs2) cy, cx (cy^2-cs2),     */
/*   (cx^2-cs2)(cy^2-cs2).                                                   */
/* M^-1 is obtained by Gauss-Jordan elimination of M, not by a formula.       */
/* ------------------------------------------------------------------------ */
typedef struct {
    double M[9][9];
    double Minv[9][9];
    double gnorm[3]; /* sum_i w_i H_g(c_i)^2 for the three ghost rows */
} mrt_t;

static double hermite_row(int a, double cx, double cy)
{
    switch (a) {
    case 0: return 1.0;
    case 1: return cx;
    case 2: return cy;
    case 3: return cx * cx - cs2;
    case 4: return cx * cy;
    case 5: return cy * cy - cs2;
    case 6: return (cx * cx - cs2) * cy;
    case 7: return cx * (cy * cy - cs2);
    default: return (cx * cx - cs2) * (cy * cy - cs2);
    }
}

static int invert9(const double A[9][9], double R[9][9])
{
    double T[9][18];
    int r, c, k;
    for (r = 0; r < 9; ++r)
        for (c = 0; c < 18; ++c) T[r][c] = (c < 9) ? A[r][c] : (c - 9 == r ? 1.0 : 0.0);
    for (c = 0; c < 9; ++c) {
        int piv = c;
        for (r = c + 1; r < 9; ++r) if (fabs(T[r][c]) > fabs(T[piv][c])) piv = r;
        if (fabs(T[piv][c]) < 1e-14) return ORA_ERR_ARG;
        if (piv != c) for (k = 0; k < 18; ++k) { double t = T[c][k]; T[c][k] = T[piv][k]; T[piv][k] = t; }
        {
            double p = T[c][c];
            for (k = 0; k < 18; ++k) T[c][k] /= p;
        }
        for (r = 0; r < 9; ++r) {
            if (r == c) continue;
            double fct = T[r][c];
            for (k = 0; k < 18; ++k) T[r][k] -= fct * T[c][k];
        }
    }
    for (r = 0; r < 9; ++r) for (c = 0; c < 9; ++c) R[r][c] = T[r][c + 9];
    return ORA_OK;
}

static int mrt_setup(const stencil_t* s, mrt_t* m)
{
    int a, i;
    if (s->q != 9) return ORA_ERR_ARG;
    for (a = 0; a < 9; ++a)
        for (i = 0; i < 9; ++i) m->M[a][i] = hermite_row(a, s->c[i][0], s->c[i][1]);
    if (invert9(m->M, m->Minv)) return ORA_ERR_ARG;
    for (a = 0; a < 3; ++a) {
        double acc = 0.0;
        for (i = 0; i < 9; ++i) acc += s->w[i] * m->M[6 + a][i] * m->M[6 + a][i];
        m->gnorm[a] = acc;
    }
    return ORA_OK;
}

/* ------------------------------------------------------------------------ */
/* The per-node network (Sec. 3.1): inputs are six rotation- and reflection- */
/* invariant combinations of the local moments, standardised by a fixed      */
/* shift and scale; two tanh layers of 24 units; one output z; the higher-   */
/* moment relaxation time is tau_g = exp(z) + 1/2, i.e. omega_g in (0, 2).    */
/* mlp layout: W1[24][6], b1[24], W2[24][24], b2[24], W3[24], b3, shift[6],   */
/* scale[6].                                                                  */
/* ------------------------------------------------------------------------ */
typedef struct {
    double x[NIN];
    double h1[NH], h2[NH];
    double z;
} mlp_cache_t;

static double mlp_forward(const double* p, const double* inv, mlp_cache_t* cc)
{
    const double *W1 = p, *b1 = W1 + NH * NIN, *W2 = b1 + NH, *b2 = W2 + NH * NH, *W3 = b2 + NH,
                 *b3 = W3 + NH, *shift = b3 + 1, *scale = shift + NIN;
    int j, k;
    double z;
    for (k = 0; k < NIN; ++k) cc->x[k] = (inv[k] - shift[k]) * scale[k];
    for (j = 0; j < NH; ++j) {
        double a = b1[j];
        for (k = 0; k < NIN; ++k) a += W1[j * NIN + k] * cc->x[k];
        cc->h1[j] = tanh(a);
    }
    for (j = 0; j < NH; ++j) {
        double a = b2[j];
        for (k = 0; k < NH; ++k) a += W2[j * NH + k] * cc->h1[k];
        cc->h2[j] = tanh(a);
    }
    z = b3[0];
    for (k = 0; k < NH; ++k) z += W3[k] * cc->h2[k];
    cc->z = z;
    return z;
}

/* The one-hidden-layer network of Sec. 3.1's description: the same six standardised
 * inputs, NH3 tanh units, three outputs z[0..2]; tau_n = exp(z_n) + 1/2 for the higher
 * moments in the order the paper lists them, N (4th order, our row 8) and J = (J0, J1)
 * (3rd order, our rows 6 and 7). Layout: W1[NH3][6], b1[NH3], W2[3][NH3], b2[3],
 * shift[6], scale[6]. */
typedef struct {
    double x[NIN];
    double h[NH3];
    double z[3];
} mlp3_cache_t;

static void mlp3_forward(const double* p, const double* inv, mlp3_cache_t* cc)
{
    const double *W1 = p, *b1 = W1 + NH3 * NIN, *W2 = b1 + NH3, *b2 = W2 + 3 * NH3, *shift = b2 + 3,
                 *scale = shift + NIN;
    int j, k, o;
    for (k = 0; k < NIN; ++k) cc->x[k] = (inv[k] - shift[k]) * scale[k];
    for (j = 0; j < NH3; ++j) {
        double a = b1[j];
        for (k = 0; k < NIN; ++k) a += W1[j * NIN + k] * cc->x[k];
        cc->h[j] = tanh(a);
    }
    for (o = 0; o < 3; ++o) {
        double a = b2[o];
        for (j = 0; j < NH3; ++j) a += W2[o * NH3 + j] * cc->h[j];
        cc->z[o] = a;
    }
}

/* ghost row (6, 7, 8) of each output of the three-output network: N -> 8, J0 -> 6, J1 -> 7 */
static const int out_row[3] = {8, 6, 7};

/* invariants of the local state used as network inputs:
 *  I1 = rho - 1, I2 = |u|^2/cs2, I3 = tr Pi^neq / cs2, I4 = Pi^neq:Pi^neq / cs2^2,
 *  I5 = u.Pi^neq.u / cs2^2, I6 = sum_g (m_g - m_g^eq)^2 / |H_g|_w^2.
 * Pi^neq and the ghost moments come from m = M f and m^eq = M f^eq. */
static void invariants(const mrt_t* mt, double rho, const double* u, const double* m, const double* meq,
                       double* I)
{
    double pxx = m[3] - meq[3], pxy = m[4] - meq[4], pyy = m[5] - meq[5];
    int g;
    I[0] = rho - 1.0;
    I[1] = (u[0] * u[0] + u[1] * u[1]) / cs2;
    I[2] = (pxx + pyy) / cs2;
    I[3] = (pxx * pxx + 2.0 * pxy * pxy + pyy * pyy) / (cs2 * cs2);
    I[4] = (u[0] * u[0] * pxx + 2.0 * u[0] * u[1] * pxy + u[1] * u[1] * pyy) / (cs2 * cs2);
    I[5] = 0.0;
    for (g = 0; g < 3; ++g) I[5] += (m[6 + g] - meq[6 + g]) * (m[6 + g] - meq[6 + g]) / mt->gnorm[g];
}

/* ------------------------------------------------------------------------ */
/* Collision of one node: f -> f* (post-collision), per collision kind.      */
/* ------------------------------------------------------------------------ */
typedef struct {
    const stencil_t* s;
    double tau;
    int coll;
    const double* mlp; /* NMLP doubles, learned collision only */
    const mrt_t* mt;   /* learned collision and MRT only */
    double tau_minus;  /* TRT: relaxation time of the antisymmetric part */
    double tau_g[3];   /* MRT: relaxation times of the three higher (ghost) moments */
} params_t;

/* 1D functions dual to the monomials 1, c, c^2 on the nodes c in {-1, 0, 1}:
 * sum_c c^b phi_a(c) = (a == b). Their products give, on D2Q9 and D3Q27 (full
 * tensor-product sets), the population vector that carries exactly one natural
 * (raw) moment sum_i cx^a cy^b cz^c f_i and none of the others. */
static double phi1d(int a, int c)
{
    if (a == 0) return c == 0 ? 1.0 : 0.0;
    if (a == 1) return 0.5 * c;
    return c == 0 ? -1.0 : 0.5;
}

static void collide_node(const params_t* P, const double* f, const double* F, double* out)
{
    const stencil_t* s = P->s;
    double omega = 1.0 / P->tau, rho, u[3], feq[27], S[27];
    int i, a, b;
    if (P->coll == ORA_NONE) {
        for (i = 0; i < s->q; ++i) out[i] = f[i];
        return;
    }
    node_moments(s, f, F, &rho, u);
    equilibrium(s, rho, u, feq);
    if (F) guo_source(s, omega, u, F, S);
    else for (i = 0; i < s->q; ++i) S[i] = 0.0;

    if (P->coll == ORA_BGK) {
        /* Eq. 2: f* = f - (f - f^eq)/tau, plus the source */
        for (i = 0; i < s->q; ++i) out[i] = f[i] - omega * (f[i] - feq[i]) + S[i];
    } else if (P->coll == ORA_REG) {
        /* Regularized: project f^neq = f - f^eq onto the Hermite polynomials of order <= 2,
         *   a1 = sum_i c_i f^neq_i (zero without a force, -F/2 with the half-force shift),
         *   Pi = sum_i c_i c_i f^neq_i,
         * and relax only that projection:
         *   f* = f^eq + (1 - omega) w_i [ c_i . a1 / cs2 + (c_i c_i - cs2 I) : Pi / (2 cs2^2) ] + S */
        double Pi[3][3] = {{0}}, a1[3] = {0};
        for (a = 0; a < s->d; ++a) {
            double acc = 0.0;
            for (i = 0; i < s->q; ++i) acc += s->c[i][a] * (f[i] - feq[i]);
            a1[a] = acc;
            for (b = 0; b < s->d; ++b) {
                acc = 0.0;
                for (i = 0; i < s->q; ++i) acc += s->c[i][a] * s->c[i][b] * (f[i] - feq[i]);
                Pi[a][b] = acc;
            }
        }
        for (i = 0; i < s->q; ++i) {
            double qp = 0.0, ca = 0.0;
            for (a = 0; a < s->d; ++a) {
                ca += s->c[i][a] * a1[a];
                for (b = 0; b < s->d; ++b)
                    qp += (s->c[i][a] * s->c[i][b] - (a == b ? cs2 : 0.0)) * Pi[a][b];
            }
            out[i] = feq[i] + (1.0 - omega) * s->w[i] * (ca / cs2 + qp / (2.0 * cs2 * cs2)) + S[i];
        }
    } else if (P->coll == ORA_TRT) {
        /* Two-relaxation-time model (Ginzburg 2008): split every population pair (i, opp i)
         * into its symmetric and antisymmetric halves,
         *   g+_i = (g_i + g_opp(i))/2,  g-_i = (g_i - g_opp(i))/2,
         * relax the symmetric non-equilibrium part with 1/tau (which sets the viscosity)
         * and the antisymmetric one with 1/tau_minus, and split the Guo source the same
         * way with prefactors (1 - omega+/2) and (1 - omega-/2):
         *   f*_i = f_i - (f+_i - feq+_i)/tau - (f-_i - feq-_i)/tau_minus
         *          + (1 - 1/(2 tau)) S+_i + (1 - 1/(2 tau_minus)) S-_i.
         * tau_minus follows from the "magic" product Lambda = (tau - 1/2)(tau_minus - 1/2). */
        double om_p = 1.0 / P->tau, om_m = 1.0 / P->tau_minus, S0[27];
        if (F) {
            /* S0 = the source without its prefactor (guo_source with omega = 0) */
            guo_source(s, 0.0, u, F, S0);
        } else {
            for (i = 0; i < s->q; ++i) S0[i] = 0.0;
        }
        for (i = 0; i < s->q; ++i) {
            int o = s->opp[i];
            double fp = 0.5 * (f[i] + f[o]), fm = 0.5 * (f[i] - f[o]);
            double ep = 0.5 * (feq[i] + feq[o]), em = 0.5 * (feq[i] - feq[o]);
            double sp = 0.5 * (S0[i] + S0[o]), sm = 0.5 * (S0[i] - S0[o]);
            out[i] = f[i] - om_p * (fp - ep) - om_m * (fm - em) + (1.0 - 0.5 * om_p) * sp + (1.0 - 0.5 * om_m) * sm;
        }
    } else if (P->coll == ORA_KBC) {
        /* Entropic KBC model (Karlin, Boesch & Chikatamarla 2014), no force, D2Q9 / D3Q27.
         * f = k + s + h in natural (raw) moments: k carries rho and rho u, s the deviatoric
         * (trace-free) second moments, h everything else (trace, third and higher orders).
         * With D = f - f^eq: Ds = the population vector whose natural moments are the
         * deviatoric second moments of D (and no other), Dh = D - Ds (Dk = 0). Then
         *   f* = f - beta (2 Ds + gamma Dh),  beta = 1/(2 tau),
         *   gamma = 1/beta - (2 - 1/beta) <Ds|Dh> / <Dh|Dh>,  <X|Y> = sum_i X_i Y_i / feq_i,
         * the gamma that minimises the quadratic entropy estimate <D*|D*> of the result.
         * Reading: the ratio's denominator is <Dh|Dh> + 1e-6 <Ds|Ds>. As Dh -> 0 along a
         * fixed direction the unregularised gamma Dh tends to a finite, direction-dependent
         * limit, so rounding noise in a vanishing Dh would decide the result; the term
         * keeps gamma Dh -> 0 there and changes gamma by a relative 1e-6 <Ds|Ds>/<Dh|Dh>
         * elsewhere. gamma = 2 (plain BGK) when D = 0. */
        double D[27], Ds[27], M2[3][3], tr = 0.0, sh = 0.0, hh = 0.0, ss = 0.0, beta = 0.5 / P->tau, gam, den;
        for (i = 0; i < s->q; ++i) D[i] = f[i] - feq[i];
        for (a = 0; a < s->d; ++a)
            for (b = 0; b < s->d; ++b) {
                double acc = 0.0;
                for (i = 0; i < s->q; ++i) acc += s->c[i][a] * s->c[i][b] * D[i];
                M2[a][b] = acc;
            }
        for (a = 0; a < s->d; ++a) tr += M2[a][a];
        for (a = 0; a < s->d; ++a) M2[a][a] -= tr / s->d;
        for (i = 0; i < s->q; ++i) {
            double acc = 0.0;
            for (a = 0; a < s->d; ++a)
                for (b = 0; b < s->d; ++b) {
                    /* exponents of the monomial c_a c_b in each axis */
                    int e[3] = {0, 0, 0}, k;
                    double prod = 1.0;
                    if (b < a) continue; /* each off-diagonal moment once */
                    e[a] += 1; e[b] += 1;
                    for (k = 0; k < 3; ++k) prod *= phi1d(e[k], s->c[i][k]);
                    acc += M2[a][b] * prod;
                }
            Ds[i] = acc;
        }
        for (i = 0; i < s->q; ++i) {
            double h = D[i] - Ds[i];
            sh += Ds[i] * h / feq[i];
            hh += h * h / feq[i];
            ss += Ds[i] * Ds[i] / feq[i];
        }
        den = hh + 1e-6 * ss;
        gam = den > 0.0 ? 1.0 / beta - (2.0 - 1.0 / beta) * sh / den : 2.0;
        for (i = 0; i < s->q; ++i) out[i] = f[i] - beta * (2.0 * Ds[i] + gam * (D[i] - Ds[i]));
    } else if (P->coll == ORA_MRT) {
        /* Eq. 5 with fixed rates: conserved rows 1, stress rows 1/tau, the three higher
         * (ghost) rows 1/tau_g[k]; D2Q9, no force. */
        const mrt_t* mt = P->mt;
        double m[9], meq[9], om[9];
        for (a = 0; a < 9; ++a) {
            double rate = a < 3 ? 1.0 : (a < 6 ? 1.0 / P->tau : 1.0 / P->tau_g[a - 6]);
            m[a] = 0.0; meq[a] = 0.0;
            for (i = 0; i < 9; ++i) { m[a] += mt->M[a][i] * f[i]; meq[a] += mt->M[a][i] * feq[i]; }
            om[a] = rate * (m[a] - meq[a]);
        }
        for (i = 0; i < 9; ++i) {
            double acc = 0.0;
            for (a = 0; a < 9; ++a) acc += mt->Minv[i][a] * om[a];
            out[i] = f[i] - acc;
        }
    } else { /* ORA_LEARNED / ORA_LEARNED3, D2Q9, no force: Eq. 5 */
        const mrt_t* mt = P->mt;
        double m[9], meq[9], rate[9], I[NIN], om[9];
        for (a = 0; a < 9; ++a) {
            m[a] = 0.0; meq[a] = 0.0;
            for (i = 0; i < 9; ++i) { m[a] += mt->M[a][i] * f[i]; meq[a] += mt->M[a][i] * feq[i]; }
        }
        invariants(mt, rho, u, m, meq, I);
        for (a = 0; a < 3; ++a) rate[a] = 1.0;          /* conserved: tau = 1 */
        for (a = 3; a < 6; ++a) rate[a] = 1.0 / P->tau; /* stress: tau_n = nu/cs2 + 1/2 */
        if (P->coll == ORA_LEARNED) {
            mlp_cache_t cc;
            double taug = exp(mlp_forward(P->mlp, I, &cc)) + 0.5;
            for (a = 6; a < 9; ++a) rate[a] = 1.0 / taug; /* higher moments from the network */
        } else {
            mlp3_cache_t c3;
            int o;
            mlp3_forward(P->mlp, I, &c3);
            for (o = 0; o < 3; ++o) rate[out_row[o]] = 1.0 / (exp(c3.z[o]) + 0.5);
        }
        for (a = 0; a < 9; ++a) om[a] = rate[a] * (m[a] - meq[a]);
        for (i = 0; i < 9; ++i) {
            double acc = 0.0;
            for (a = 0; a < 9; ++a) acc += mt->Minv[i][a] * om[a];
            out[i] = f[i] - acc;
        }
    }
}

/* cpar: the collision's parameters. Learned: the NMLP network values. TRT: cpar[0] =
 * Lambda (default 1/4 when cpar is NULL). MRT: cpar[0..2] = tau_g of the three higher
 * moments (default 1 each). Others: unused. */
static int make_params(params_t* P, const stencil_t* s, mrt_t* mt, double tau, int coll, const double* cpar,
                       const double* F)
{
    int k;
    P->s = s; P->tau = tau; P->coll = coll; P->mlp = NULL; P->mt = NULL;
    P->tau_minus = tau;
    P->tau_g[0] = P->tau_g[1] = P->tau_g[2] = 1.0;
    if (!(tau > 0.5)) return ORA_ERR_ARG;
    if (coll < 0 || coll > 7) return ORA_ERR_ARG;
    if (coll == ORA_LEARNED || coll == ORA_LEARNED3) {
        if (s->q != 9 || !cpar || F) return ORA_ERR_ARG;
        if (mrt_setup(s, mt)) return ORA_ERR_ARG;
        P->mlp = cpar;
        P->mt = mt;
    } else if (coll == ORA_TRT) {
        double lam = cpar ? cpar[0] : 0.25;
        if (!(lam > 0.0)) return ORA_ERR_ARG;
        P->tau_minus = 0.5 + lam / (tau - 0.5);
    } else if (coll == ORA_KBC) {
        if (F || (s->q != 9 && s->q != 27)) return ORA_ERR_ARG;
    } else if (coll == ORA_MRT) {
        if (s->q != 9 || F) return ORA_ERR_ARG;
        if (mrt_setup(s, mt)) return ORA_ERR_ARG;
        P->mt = mt;
        if (cpar)
            for (k = 0; k < 3; ++k) {
                if (!(cpar[k] > 0.5)) return ORA_ERR_ARG;
                P->tau_g[k] = cpar[k];
            }
    }
    return ORA_OK;
}

int ora_collide_node(int st, double tau, int coll, const double* f, const double* F, const double* mlp,
                     double* out)
{
    stencil_t s;
    mrt_t mt;
    params_t P;
    double FF[3] = {0, 0, 0};
    if (stencil_get(st, &s)) return ORA_ERR_ARG;
    if (F) { FF[0] = F[0]; FF[1] = F[1]; if (s.d == 3) FF[2] = F[2]; }
    if (make_params(&P, &s, &mt, tau, coll, mlp, F)) return ORA_ERR_ARG;
    collide_node(&P, f, F ? FF : NULL, out);
    return ORA_OK;
}

/* gather / scatter of one node of a [Q][N] array */
static void gather(const stencil_t* s, const double* f, int64_t N, int64_t n, double* fl)
{
    int i;
    for (i = 0; i < s->q; ++i) fl[i] = f[(int64_t)i * N + n];
}

static void node_force(const stencil_t* s, const double* F, int64_t N, int64_t n, double* Fl)
{
    int a;
    Fl[0] = Fl[1] = Fl[2] = 0.0;
    for (a = 0; a < s->d; ++a) Fl[a] = F[(int64_t)a * N + n];
}

/* ------------------------------------------------------------------------ */
/* Eq. 1 time stepping: collide every node, then push f*_i to x + c_i.       */
/* f is the pre-collision state f^n[Q][N] and is replaced by f^{n+steps}.    */
/* ------------------------------------------------------------------------ */
int ora_step(int st, const int64_t* dims, double tau, int coll, const double* F, const double* mlp, double* f,
             int64_t nsteps)
{
    stencil_t s;
    mrt_t mt;
    params_t P;
    int64_t N, t, n;
    double* g;
    if (stencil_get(st, &s) || check_dims(&s, dims)) return ORA_ERR_ARG;
    if (make_params(&P, &s, &mt, tau, coll, mlp, F)) return ORA_ERR_ARG;
    N = dims[0] * dims[1] * dims[2];
    g = (double*)malloc(sizeof(double) * (size_t)s.q * (size_t)N);
    if (!g) return ORA_ERR_OOM;
    for (t = 0; t < nsteps; ++t) {
#pragma omp parallel for schedule(static)
        for (n = 0; n < N; ++n) {
            double fl[27], out[27], Fl[3];
            int i;
            gather(&s, f, N, n, fl);
            if (F) node_force(&s, F, N, n, Fl);
            collide_node(&P, fl, F ? Fl : NULL, out);
            for (i = 0; i < s.q; ++i)
                g[(int64_t)i * N + shifted_node(dims, n, s.c[i][0], s.c[i][1], s.c[i][2])] = out[i];
        }
        memcpy(f, g, sizeof(double) * (size_t)s.q * (size_t)N);
    }
    free(g);
    return ORA_OK;
}

/* ------------------------------------------------------------------------ */
/* Velocity-shift forcing of Sec. 3.2: a BGK step (Eq. 2) whose equilibrium   */
/* is expanded around the locally shifted velocity u + du,                    */
/*   f*_i = f_i - (f_i - f^eq_i(rho, u + du)) / tau,  u = sum_i c_i f_i / rho, */
/* then streaming as in ora_step. du[d][N] is given (held fixed over the      */
/* nsteps steps; Sec. 3.2 recomputes it from the state every step).           */
/* ------------------------------------------------------------------------ */
int ora_step_ushift(int st, const int64_t* dims, double tau, const double* du, double* f, int64_t nsteps)
{
    stencil_t s;
    int64_t N, t, n;
    double* g;
    if (stencil_get(st, &s) || check_dims(&s, dims) || !du || !(tau > 0.5)) return ORA_ERR_ARG;
    N = dims[0] * dims[1] * dims[2];
    g = (double*)malloc(sizeof(double) * (size_t)s.q * (size_t)N);
    if (!g) return ORA_ERR_OOM;
    for (t = 0; t < nsteps; ++t) {
#pragma omp parallel for schedule(static)
        for (n = 0; n < N; ++n) {
            double fl[27], feq[27], rho, u[3], us[3], omega = 1.0 / tau;
            int i, a;
            gather(&s, f, N, n, fl);
            node_moments(&s, fl, NULL, &rho, u);
            for (a = 0; a < 3; ++a) us[a] = u[a] + (a < s.d ? du[(int64_t)a * N + n] : 0.0);
            equilibrium(&s, rho, us, feq);
            for (i = 0; i < s.q; ++i)
                g[(int64_t)i * N + shifted_node(dims, n, s.c[i][0], s.c[i][1], s.c[i][2])] =
                    fl[i] - omega * (fl[i] - feq[i]);
        }
        memcpy(f, g, sizeof(double) * (size_t)s.q * (size_t)N);
    }
    free(g);
    return ORA_OK;
}

/* ------------------------------------------------------------------------ */
/* Eq. 1 with solid nodes: halfway bounce-back (the paper lists boundary      */
/* conditions without formulas, Sec. 2.2; textbook form, Krueger et al. 2016, */
/* Ladd's moving-wall term). A fluid node collides and pushes f*_i to x + c_i; */
/* where x + c_i is solid, the population returns to x in the opposite slot:  */
/*   f_opp(i)(x, t + 1) = f*_i(x, t) - 2 w_i (c_i . u_w) / c_s^2,             */
/* with u_w the wall velocity stored at the solid node x + c_i (wall density  */
/* taken as 1). Solid nodes do not collide; they hold the rest equilibrium    */
/* w_i. mask[N]: nonzero = solid. wall_u[3][N] (or NULL = resting walls).     */
/* ------------------------------------------------------------------------ */
int ora_step_walls(int st, const int64_t* dims, double tau, int coll, const double* F, const double* cpar,
                   const unsigned char* mask, const double* wall_u, double* f, int64_t nsteps)
{
    stencil_t s;
    mrt_t mt;
    params_t P;
    int64_t N, t, n;
    double* g;
    if (!mask) return ORA_ERR_ARG;
    if (stencil_get(st, &s) || check_dims(&s, dims)) return ORA_ERR_ARG;
    if (make_params(&P, &s, &mt, tau, coll, cpar, F)) return ORA_ERR_ARG;
    N = dims[0] * dims[1] * dims[2];
    g = (double*)malloc(sizeof(double) * (size_t)s.q * (size_t)N);
    if (!g) return ORA_ERR_OOM;
    for (t = 0; t < nsteps; ++t) {
#pragma omp parallel for schedule(static)
        for (n = 0; n < N; ++n) {
            double fl[27], out[27], Fl[3];
            int i, a;
            if (mask[n]) {
                for (i = 0; i < s.q; ++i) g[(int64_t)i * N + n] = s.w[i];
                continue;
            }
            gather(&s, f, N, n, fl);
            if (F) node_force(&s, F, N, n, Fl);
            collide_node(&P, fl, F ? Fl : NULL, out);
            for (i = 0; i < s.q; ++i) {
                int64_t y = shifted_node(dims, n, s.c[i][0], s.c[i][1], s.c[i][2]);
                if (mask[y]) {
                    double cu = 0.0;
                    if (wall_u)
                        for (a = 0; a < s.d; ++a) cu += s.c[i][a] * wall_u[(int64_t)a * N + y];
                    g[(int64_t)s.opp[i] * N + n] = out[i] - 2.0 * s.w[i] * cu / cs2;
                } else {
                    g[(int64_t)i * N + y] = out[i];
                }
            }
        }
        memcpy(f, g, sizeof(double) * (size_t)s.q * (size_t)N);
    }
    free(g);
    return ORA_OK;
}

/* f_i = f_i^eq(rho, u) at every node (equilibrium initialisation) */
int ora_init_eq(int st, const int64_t* dims, const double* rho, const double* u, double* f)
{
    stencil_t s;
    int64_t N, n;
    int i, a;
    if (stencil_get(st, &s) || check_dims(&s, dims)) return ORA_ERR_ARG;
    N = dims[0] * dims[1] * dims[2];
    for (n = 0; n < N; ++n) {
        double ul[3] = {0, 0, 0}, feq[27];
        for (a = 0; a < s.d; ++a) ul[a] = u[(int64_t)a * N + n];
        equilibrium(&s, rho[n], ul, feq);
        for (i = 0; i < s.q; ++i) f[(int64_t)i * N + n] = feq[i];
    }
    return ORA_OK;
}

/* density and velocity of the (pre-collision) state, u with the half-force shift */
int ora_moments(int st, const int64_t* dims, const double* F, const double* f, double* rho, double* u)
{
    stencil_t s;
    int64_t N, n;
    int a;
    if (stencil_get(st, &s) || check_dims(&s, dims)) return ORA_ERR_ARG;
    N = dims[0] * dims[1] * dims[2];
    for (n = 0; n < N; ++n) {
        double fl[27], Fl[3], r, ul[3];
        gather(&s, f, N, n, fl);
        if (F) node_force(&s, F, N, n, Fl);
        node_moments(&s, fl, F ? Fl : NULL, &r, ul);
        rho[n] = r;
        for (a = 0; a < s.d; ++a) u[(int64_t)a * N + n] = ul[a];
    }
    return ORA_OK;
}

/* global sums in node order: out = {sum rho, sum rho u_x, sum rho u_y, sum rho u_z,
 * (1/2N) sum |u|^2 (incompressible kinetic energy), (1/2N) sum rho |u|^2} */
int ora_reduce(int st, const int64_t* dims, const double* F, const double* f, double* out)
{
    stencil_t s;
    int64_t N, n;
    int a;
    double acc[6] = {0, 0, 0, 0, 0, 0};
    if (stencil_get(st, &s) || check_dims(&s, dims)) return ORA_ERR_ARG;
    N = dims[0] * dims[1] * dims[2];
    for (n = 0; n < N; ++n) {
        double fl[27], Fl[3], r, ul[3], uu;
        gather(&s, f, N, n, fl);
        if (F) node_force(&s, F, N, n, Fl);
        node_moments(&s, fl, F ? Fl : NULL, &r, ul);
        uu = ul[0] * ul[0] + ul[1] * ul[1] + ul[2] * ul[2];
        acc[0] += r;
        for (a = 0; a < 3; ++a) acc[1 + a] += r * ul[a];
        acc[4] += uu;
        acc[5] += r * uu;
    }
    for (a = 0; a < 4; ++a) out[a] = acc[a];
    out[4] = 0.5 * acc[4] / (double)N;
    out[5] = 0.5 * acc[5] / (double)N;
    return ORA_OK;
}

/* the network's relaxation rate omega_g = 1 / (exp(z) + 1/2) for given invariants */
int ora_mlp_omega(const double* mlp, const double* I, double* omega)
{
    mlp_cache_t cc;
    double z = mlp_forward(mlp, I, &cc);
    *omega = 1.0 / (exp(z) + 0.5);
    return ORA_OK;
}

/* the six network inputs of one D2Q9 node (for tests) */
int ora_invariants(const double* f, double* I)
{
    stencil_t s;
    mrt_t mt;
    double rho, u[3], feq[9], m[9], meq[9];
    int a, i;
    stencil_get(0, &s);
    if (mrt_setup(&s, &mt)) return ORA_ERR_ARG;
    node_moments(&s, f, NULL, &rho, u);
    equilibrium(&s, rho, u, feq);
    for (a = 0; a < 9; ++a) {
        m[a] = 0.0; meq[a] = 0.0;
        for (i = 0; i < 9; ++i) { m[a] += mt.M[a][i] * f[i]; meq[a] += mt.M[a][i] * feq[i]; }
    }
    invariants(&mt, rho, u, m, meq, I);
    return ORA_OK;
}

/* ======================================================================== */
/* Discrete adjoint (Sec. 3.2 takes gradients through the solver; here the   */
/* transposed Jacobian of each step is written out by the chain rule).       */
/* One step is f^{n+1} = S C(f^n; F) with S the periodic shift by c_i. Its   */
/* transpose: mu_i(x) = lambda^{n+1}_i(x + c_i); lambda^n(x) = J_C(x)^T mu(x); */
/* dL/dF(x) += (dC/dF)^T mu(x); dL/dtheta += (dC/dtheta)^T mu(x).             */
/* ======================================================================== */

/* d f^eq_i / d rho and d f^eq_i / d u (closed form of Eq. 3's derivative) */
static void feq_derivs(const stencil_t* s, double rho, const double* u, double* drho, double (*du)[3])
{
    int i, a;
    double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    for (i = 0; i < s->q; ++i) {
        double cu = s->c[i][0] * u[0] + s->c[i][1] * u[1] + s->c[i][2] * u[2];
        drho[i] = s->w[i] * (1.0 + cu / cs2 + cu * cu / (2.0 * cs2 * cs2) - uu / (2.0 * cs2));
        for (a = 0; a < 3; ++a)
            du[i][a] = s->w[i] * rho * (s->c[i][a] / cs2 + cu * s->c[i][a] / (cs2 * cs2) - u[a] / cs2);
    }
}

/* One node of the transposed collision Jacobian.
 * in: f (pre-collision node state), F (or NULL), mu (cotangent of f*)
 * out: lam = J^T mu; gF += (dC/dF)^T mu; gth += (dC/dtheta)^T mu (learned only) */
static void adjoint_node(const params_t* P, const double* f, const double* F, const double* mu, double* lam,
                         double* gF, double* gth)
{
    const stencil_t* s = P->s;
    double omega = 1.0 / P->tau, rho, u[3], drho[27], du[27][3];
    double grho = 0.0, gu[3] = {0, 0, 0}; /* cotangents of rho and u (excluding the direct path) */
    double gFl[3] = {0, 0, 0};
    int i, a, b;
    if (P->coll == ORA_NONE) {
        for (i = 0; i < s->q; ++i) lam[i] = mu[i];
        return;
    }
    node_moments(s, f, F, &rho, u);
    feq_derivs(s, rho, u, drho, du);

    if (P->coll == ORA_BGK) {
        /* f*_i = (1 - omega) f_i + omega f^eq_i(rho, u) + S_i(u, F) */
        for (i = 0; i < s->q; ++i) {
            lam[i] = (1.0 - omega) * mu[i];
            grho += mu[i] * omega * drho[i];
            for (a = 0; a < 3; ++a) gu[a] += mu[i] * omega * du[i][a];
        }
    } else if (P->coll == ORA_REG) {
        /* f*_i = f^eq_i + h_i [ c_i . a1 / cs2 + Q_i : Pi / (2 cs2) ] + S_i,  h_i = (1 - omega) w_i / cs2,
         * with Pi = sum_k c_k c_k f_k - (rho u u + rho cs2 I) and a1 = j - rho u = -F/2.
         * G = sum_i mu_i (1 - omega) w_i Q_i / (2 cs2^2) is the cotangent of Pi,
         * A = sum_i mu_i (1 - omega) w_i c_i / cs2 the cotangent of a1. */
        double G[3][3] = {{0}}, A[3] = {0};
        for (a = 0; a < s->d; ++a) {
            double acc = 0.0;
            for (i = 0; i < s->q; ++i) acc += mu[i] * (1.0 - omega) * s->w[i] * s->c[i][a] / cs2;
            A[a] = acc;
            for (b = 0; b < s->d; ++b) {
                acc = 0.0;
                for (i = 0; i < s->q; ++i)
                    acc += mu[i] * (1.0 - omega) * s->w[i] / (2.0 * cs2 * cs2) *
                           (s->c[i][a] * s->c[i][b] - (a == b ? cs2 : 0.0));
                G[a][b] = acc;
            }
        }
        for (i = 0; i < s->q; ++i) {
            double cgc = 0.0;
            for (a = 0; a < s->d; ++a)
                for (b = 0; b < s->d; ++b) cgc += s->c[i][a] * G[a][b] * s->c[i][b];
            lam[i] = cgc; /* direct path through sum_k c_k c_k f_k */
            grho += mu[i] * drho[i];
            for (a = 0; a < s->d; ++a) gu[a] += mu[i] * du[i][a];
        }
        {
            double uGu = 0.0, trG = 0.0, Gu[3] = {0, 0, 0};
            for (a = 0; a < s->d; ++a) {
                trG += G[a][a];
                for (b = 0; b < s->d; ++b) {
                    uGu += u[a] * G[a][b] * u[b];
                    Gu[a] += G[a][b] * u[b];
                }
            }
            grho -= uGu + cs2 * trG;
            for (a = 0; a < s->d; ++a) {
                gu[a] += -2.0 * rho * Gu[a];
                if (F) gFl[a] += -0.5 * A[a]; /* a1 = -F/2 */
            }
        }
    } else { /* learned Eq. 5 (one shared or three separate higher-moment rates), D2Q9, no force */
        const mrt_t* mt = P->mt;
        const double* p = P->mlp;
        double feq[9], m[9], meq[9], I[NIN], nu[9], gm[9], gI[NIN], gx[NIN];
        double rate_g[3], ez_g[3], kap[3], gP[3];
        mlp_cache_t cc;
        mlp3_cache_t c3;
        int j, k, o;
        equilibrium(s, rho, u, feq);
        for (a = 0; a < 9; ++a) {
            m[a] = 0.0; meq[a] = 0.0;
            for (i = 0; i < 9; ++i) { m[a] += mt->M[a][i] * f[i]; meq[a] += mt->M[a][i] * feq[i]; }
        }
        invariants(mt, rho, u, m, meq, I);
        if (P->coll == ORA_LEARNED) {
            double ez = exp(mlp_forward(p, I, &cc));
            for (a = 0; a < 3; ++a) { ez_g[a] = ez; rate_g[a] = 1.0 / (ez + 0.5); }
        } else {
            mlp3_forward(p, I, &c3);
            for (o = 0; o < 3; ++o) {
                ez_g[out_row[o] - 6] = exp(c3.z[o]);
                rate_g[out_row[o] - 6] = 1.0 / (exp(c3.z[o]) + 0.5);
            }
        }
        /* f*_i = f_i - sum_a Minv[i][a] omega_a (m_a - meq_a); nu_a = sum_i mu_i Minv[i][a] */
        for (a = 0; a < 9; ++a) {
            nu[a] = 0.0;
            for (i = 0; i < 9; ++i) nu[a] += mu[i] * mt->Minv[i][a];
            gm[a] = 0.0;
        }
        /* stress rows: -omega_s nu_a (m_a - meq_a); meq_3 = rho ux^2, meq_4 = rho ux uy, meq_5 = rho uy^2 */
        gP[0] = -omega * nu[3]; gP[1] = -omega * nu[4]; gP[2] = -omega * nu[5];
        /* ghost rows (meq_g = 0 for the second-order equilibrium on D2Q9); kap = d L / d omega_g */
        for (a = 6; a < 9; ++a) { gm[a] += -rate_g[a - 6] * nu[a]; kap[a - 6] = -nu[a] * (m[a] - meq[a]); }
        /* omega_g = 1/(e^z + 1/2): d omega_g / dz = -e^z / (e^z + 1/2)^2 */
        if (P->coll == ORA_LEARNED) {
            const double *W1 = p, *W2 = W1 + NH * NIN + NH, *W3 = W2 + NH * NH + NH, *scale = W3 + NH + 1 + NIN;
            double *gW1 = gth, *gb1 = gW1 + NH * NIN, *gW2 = gb1 + NH, *gb2 = gW2 + NH * NH, *gW3 = gb2 + NH,
                   *gb3 = gW3 + NH;
            double ga2[NH], ga1[NH], gh1[NH], gz = 0.0;
            for (a = 0; a < 3; ++a) gz += kap[a] * (-ez_g[a] * rate_g[a] * rate_g[a]);
            /* back through the network */
            gb3[0] += gz;
            for (k = 0; k < NH; ++k) {
                gW3[k] += gz * cc.h2[k];
                ga2[k] = gz * W3[k] * (1.0 - cc.h2[k] * cc.h2[k]);
                gb2[k] += ga2[k];
            }
            for (j = 0; j < NH; ++j)
                for (k = 0; k < NH; ++k) gW2[j * NH + k] += ga2[j] * cc.h1[k];
            for (k = 0; k < NH; ++k) {
                gh1[k] = 0.0;
                for (j = 0; j < NH; ++j) gh1[k] += W2[j * NH + k] * ga2[j];
                ga1[k] = gh1[k] * (1.0 - cc.h1[k] * cc.h1[k]);
                gb1[k] += ga1[k];
            }
            for (j = 0; j < NH; ++j)
                for (k = 0; k < NIN; ++k) gW1[j * NIN + k] += ga1[j] * cc.x[k];
            for (k = 0; k < NIN; ++k) {
                gx[k] = 0.0;
                for (j = 0; j < NH; ++j) gx[k] += W1[j * NIN + k] * ga1[j];
                gI[k] = gx[k] * scale[k];
            }
        } else {
            const double *W1 = p, *W2 = W1 + NH3 * NIN + NH3, *scale = W2 + 3 * NH3 + 3 + NIN;
            double *gW1 = gth, *gb1 = gW1 + NH3 * NIN, *gW2 = gb1 + NH3, *gb2 = gW2 + 3 * NH3;
            double gz[3], ga1[NH3];
            for (o = 0; o < 3; ++o) {
                const int g = out_row[o] - 6;
                gz[o] = kap[g] * (-ez_g[g] * rate_g[g] * rate_g[g]);
                gb2[o] += gz[o];
                for (j = 0; j < NH3; ++j) gW2[o * NH3 + j] += gz[o] * c3.h[j];
            }
            for (j = 0; j < NH3; ++j) {
                double acc = 0.0;
                for (o = 0; o < 3; ++o) acc += W2[o * NH3 + j] * gz[o];
                ga1[j] = acc * (1.0 - c3.h[j] * c3.h[j]);
                gb1[j] += ga1[j];
                for (k = 0; k < NIN; ++k) gW1[j * NIN + k] += ga1[j] * c3.x[k];
            }
            for (k = 0; k < NIN; ++k) {
                gx[k] = 0.0;
                for (j = 0; j < NH3; ++j) gx[k] += W1[j * NIN + k] * ga1[j];
                gI[k] = gx[k] * scale[k];
            }
        }
        /* back through the invariants */
        {
            double pxx = m[3] - meq[3], pxy = m[4] - meq[4], pyy = m[5] - meq[5];
            grho += gI[0];
            gu[0] += 2.0 * u[0] / cs2 * gI[1];
            gu[1] += 2.0 * u[1] / cs2 * gI[1];
            gP[0] += gI[2] / cs2;
            gP[2] += gI[2] / cs2;
            gP[0] += 2.0 * pxx / (cs2 * cs2) * gI[3];
            gP[1] += 4.0 * pxy / (cs2 * cs2) * gI[3];
            gP[2] += 2.0 * pyy / (cs2 * cs2) * gI[3];
            gP[0] += u[0] * u[0] / (cs2 * cs2) * gI[4];
            gP[1] += 2.0 * u[0] * u[1] / (cs2 * cs2) * gI[4];
            gP[2] += u[1] * u[1] / (cs2 * cs2) * gI[4];
            gu[0] += (2.0 * u[0] * pxx + 2.0 * u[1] * pxy) / (cs2 * cs2) * gI[4];
            gu[1] += (2.0 * u[0] * pxy + 2.0 * u[1] * pyy) / (cs2 * cs2) * gI[4];
            for (a = 0; a < 3; ++a) gm[6 + a] += 2.0 * (m[6 + a] - meq[6 + a]) / mt->gnorm[a] * gI[5];
        }
        /* P_ab = m_{3,4,5} - meq_{3,4,5}(rho, u) */
        gm[3] += gP[0]; gm[4] += gP[1]; gm[5] += gP[2];
        grho -= gP[0] * u[0] * u[0] + gP[1] * u[0] * u[1] + gP[2] * u[1] * u[1];
        gu[0] -= gP[0] * 2.0 * rho * u[0] + gP[1] * rho * u[1];
        gu[1] -= gP[1] * rho * u[0] + gP[2] * 2.0 * rho * u[1];
        for (j = 0; j < 9; ++j) {
            double acc = mu[j];
            for (a = 0; a < 9; ++a) acc += gm[a] * mt->M[a][j];
            lam[j] = acc;
        }
    }
    /* Guo source (BGK and regularized): S_i(u, F) */
    if (F && P->coll != ORA_LEARNED && P->coll != ORA_LEARNED3) {
        for (i = 0; i < s->q; ++i) {
            double cu = s->c[i][0] * u[0] + s->c[i][1] * u[1] + s->c[i][2] * u[2];
            double cF = s->c[i][0] * F[0] + s->c[i][1] * F[1] + s->c[i][2] * F[2];
            double pre = (1.0 - 0.5 * omega) * s->w[i];
            for (a = 0; a < 3; ++a) {
                gu[a] += mu[i] * pre * (-F[a] / cs2 + cF * s->c[i][a] / (cs2 * cs2));
                gFl[a] += mu[i] * pre * ((s->c[i][a] - u[a]) / cs2 + cu * s->c[i][a] / (cs2 * cs2));
            }
        }
    }
    /* through rho (d rho / d f_j = 1) and u (d u / d f_j = (c_j - u)/rho, d u / dF = 1/(2 rho)) */
    for (i = 0; i < s->q; ++i) {
        double acc = grho;
        for (a = 0; a < 3; ++a) acc += gu[a] * (s->c[i][a] - u[a]) / rho;
        lam[i] += acc;
    }
    if (F)
        for (a = 0; a < s->d; ++a) gF[a] += gFl[a] + gu[a] / (2.0 * rho);
}

/* Adjoint of nsteps steps started from f0 (pre-collision).
 * lam: in lambda^N = dL/df^N, out lambda^0 = dL/df^0   [Q][N]
 * gF (may be NULL): += dL/dF through the steps           [d][N]
 * gth (may be NULL, learned only): += dL/dtheta          [793]
 * All intermediate states are recomputed and stored (small grids only). */
int ora_adjoint(int st, const int64_t* dims, double tau, int coll, const double* F, const double* mlp,
                const double* f0, int64_t nsteps, double* lam, double* gF, double* gth)
{
    stencil_t s;
    mrt_t mt;
    params_t P;
    int64_t N, QN, t, n;
    double *states, *mu;
    if (stencil_get(st, &s) || check_dims(&s, dims) || nsteps < 0) return ORA_ERR_ARG;
    if (coll == ORA_TRT || coll == ORA_KBC || coll == ORA_MRT) return ORA_ERR_ARG; /* no adjoint of these */
    if (make_params(&P, &s, &mt, tau, coll, mlp, F)) return ORA_ERR_ARG;
    N = dims[0] * dims[1] * dims[2];
    QN = (int64_t)s.q * N;
    states = (double*)malloc(sizeof(double) * (size_t)QN * (size_t)(nsteps > 0 ? nsteps : 1));
    mu = (double*)malloc(sizeof(double) * (size_t)QN);
    if (!states || !mu) { free(states); free(mu); return ORA_ERR_OOM; }
    if (nsteps > 0) memcpy(states, f0, sizeof(double) * (size_t)QN);
    for (t = 1; t < nsteps; ++t) {
        memcpy(states + t * QN, states + (t - 1) * QN, sizeof(double) * (size_t)QN);
        if (ora_step(st, dims, tau, coll, F, mlp, states + t * QN, 1)) { free(states); free(mu); return ORA_ERR_ARG; }
    }
    for (t = nsteps - 1; t >= 0; --t) {
        const double* fn = states + t * QN;
        /* mu_i(x) = lambda_i(x + c_i): the transpose of the shift */
        for (n = 0; n < N; ++n) {
            int i;
            for (i = 0; i < s.q; ++i)
                mu[(int64_t)i * N + n] = lam[(int64_t)i * N + shifted_node(dims, n, s.c[i][0], s.c[i][1], s.c[i][2])];
        }
        for (n = 0; n < N; ++n) {
            double fl[27], ml[27], ll[27], Fl[3], gFl[3] = {0, 0, 0};
            int i, a;
            gather(&s, fn, N, n, fl);
            gather(&s, mu, N, n, ml);
            if (F) node_force(&s, F, N, n, Fl);
            adjoint_node(&P, fl, F ? Fl : NULL, ml, ll, gFl, gth);
            for (i = 0; i < s.q; ++i) lam[(int64_t)i * N + n] = ll[i];
            if (F && gF)
                for (a = 0; a < s.d; ++a) gF[(int64_t)a * N + n] += gFl[a];
        }
    }
    free(states);
    free(mu);
    return ORA_OK;
}

/* Seed from moment cotangents: given dL/drho[N] and dL/du[d][N] of the moments of
 * state f (u with the half-force shift), lam_i = dL/drho + dL/du . (c_i - u)/rho,
 * and gF += dL/du / (2 rho) (the force enters u directly). */
int ora_seed_moments(int st, const int64_t* dims, const double* F, const double* f, const double* grho,
                     const double* gu, double* lam, double* gF)
{
    stencil_t s;
    int64_t N, n;
    if (stencil_get(st, &s) || check_dims(&s, dims)) return ORA_ERR_ARG;
    N = dims[0] * dims[1] * dims[2];
    for (n = 0; n < N; ++n) {
        double fl[27], Fl[3], r, ul[3], g[3] = {0, 0, 0};
        int i, a;
        gather(&s, f, N, n, fl);
        if (F) node_force(&s, F, N, n, Fl);
        node_moments(&s, fl, F ? Fl : NULL, &r, ul);
        for (a = 0; a < s.d; ++a) g[a] = gu[(int64_t)a * N + n];
        for (i = 0; i < s.q; ++i) {
            double acc = grho ? grho[n] : 0.0;
            for (a = 0; a < 3; ++a) acc += g[a] * (s.c[i][a] - ul[a]) / r;
            lam[(int64_t)i * N + n] = acc;
        }
        if (F && gF)
            for (a = 0; a < s.d; ++a) gF[(int64_t)a * N + n] += g[a] / (2.0 * r);
    }
    return ORA_OK;
}

/* Kinetic-energy-field loss L = sum_x (e(x) - e*(x))^2, e = rho |u|^2 / 2, and its
 * seed lambda^N = dL/df^N (and the direct force part of dL/dF through u). */
int ora_loss_energy(int st, const int64_t* dims, const double* F, const double* f, const double* etarget,
                    double* loss, double* lam, double* gF)
{
    stencil_t s;
    int64_t N, n;
    double *grho, *gu, L = 0.0;
    int rc;
    if (stencil_get(st, &s) || check_dims(&s, dims)) return ORA_ERR_ARG;
    N = dims[0] * dims[1] * dims[2];
    grho = (double*)malloc(sizeof(double) * (size_t)N);
    gu = (double*)calloc((size_t)3 * (size_t)N, sizeof(double));
    if (!grho || !gu) { free(grho); free(gu); return ORA_ERR_OOM; }
    for (n = 0; n < N; ++n) {
        double fl[27], Fl[3], r, ul[3], uu, e;
        int a;
        gather(&s, f, N, n, fl);
        if (F) node_force(&s, F, N, n, Fl);
        node_moments(&s, fl, F ? Fl : NULL, &r, ul);
        uu = ul[0] * ul[0] + ul[1] * ul[1] + ul[2] * ul[2];
        e = 0.5 * r * uu;
        L += (e - etarget[n]) * (e - etarget[n]);
        /* de/drho at fixed u = |u|^2/2, de/du = rho u */
        grho[n] = 2.0 * (e - etarget[n]) * 0.5 * uu;
        for (a = 0; a < s.d; ++a) gu[(int64_t)a * N + n] = 2.0 * (e - etarget[n]) * r * ul[a];
    }
    *loss = L;
    rc = ora_seed_moments(st, dims, F, f, grho, gu, lam, gF);
    free(grho);
    free(gu);
    return rc;
}

/* Eq. 6 training loss on a D2Q9 state (no force):
 *   L = w_u mean_x |u - u~|^2 + w_w mean_x (w - w~)^2 + w_E (E - E~)^2
 * with w_u = 0.6, w_w = w_E = 0.2, vorticity w = d_x v - d_y u by second-order
 * central differences on the periodic grid, E = (1/2N) sum |u|^2.
 * Writes L and lambda = dL/df. */
int ora_loss_eq6(const int64_t* dims, const double* f, const double* uref, const double* wref, double Eref,
                 double* loss, double* lam)
{
    stencil_t s;
    int64_t N, n;
    double *u, *rho, *w, *r, *gu, E = 0.0, Lu = 0.0, Lw = 0.0;
    const double wu = 0.6, ww = 0.2, wE = 0.2;
    int rc;
    stencil_get(0, &s);
    if (check_dims(&s, dims)) return ORA_ERR_ARG;
    N = dims[0] * dims[1];
    u = (double*)malloc(sizeof(double) * 2 * (size_t)N);
    rho = (double*)malloc(sizeof(double) * (size_t)N);
    w = (double*)malloc(sizeof(double) * (size_t)N);
    r = (double*)malloc(sizeof(double) * (size_t)N);
    gu = (double*)calloc(2 * (size_t)N, sizeof(double));
    if (!u || !rho || !w || !r || !gu) { free(u); free(rho); free(w); free(r); free(gu); return ORA_ERR_OOM; }
    ora_moments(0, dims, NULL, f, rho, u);
    for (n = 0; n < N; ++n) {
        int64_t xp = shifted_node(dims, n, 1, 0, 0), xm = shifted_node(dims, n, -1, 0, 0);
        int64_t yp = shifted_node(dims, n, 0, 1, 0), ym = shifted_node(dims, n, 0, -1, 0);
        w[n] = 0.5 * (u[N + xp] - u[N + xm]) - 0.5 * (u[yp] - u[ym]);
        E += u[n] * u[n] + u[N + n] * u[N + n];
    }
    E = 0.5 * E / (double)N;
    for (n = 0; n < N; ++n) {
        double dx = u[n] - uref[n], dy = u[N + n] - uref[N + n], dw = w[n] - wref[n];
        Lu += dx * dx + dy * dy;
        Lw += dw * dw;
        r[n] = 2.0 * ww * dw / (double)N;
        gu[n] = 2.0 * wu * dx / (double)N + 2.0 * wE * (E - Eref) * u[n] / (double)N;
        gu[N + n] = 2.0 * wu * dy / (double)N + 2.0 * wE * (E - Eref) * u[N + n] / (double)N;
    }
    *loss = wu * Lu / (double)N + ww * Lw / (double)N + wE * (E - Eref) * (E - Eref);
    /* vorticity term: w(x) = (v(x+ex) - v(x-ex))/2 - (u(x+ey) - u(x-ey))/2 */
    for (n = 0; n < N; ++n) {
        int64_t xp = shifted_node(dims, n, 1, 0, 0), xm = shifted_node(dims, n, -1, 0, 0);
        int64_t yp = shifted_node(dims, n, 0, 1, 0), ym = shifted_node(dims, n, 0, -1, 0);
        gu[N + n] += 0.5 * r[xm] - 0.5 * r[xp];
        gu[n] += -0.5 * r[ym] + 0.5 * r[yp];
    }
    rc = ora_seed_moments(0, dims, NULL, f, NULL, gu, lam, NULL);
    free(u); free(rho); free(w); free(r); free(gu);
    return rc;
}

/* Vorticity and kinetic energy of a D2Q9 state (the Eq. 6 loss targets). */
int ora_vorticity(const int64_t* dims, const double* f, double* w, double* E)
{
    stencil_t s;
    int64_t N, n;
    double *u, *rho, acc = 0.0;
    stencil_get(0, &s);
    if (check_dims(&s, dims)) return ORA_ERR_ARG;
    N = dims[0] * dims[1];
    u = (double*)malloc(sizeof(double) * 2 * (size_t)N);
    rho = (double*)malloc(sizeof(double) * (size_t)N);
    if (!u || !rho) { free(u); free(rho); return ORA_ERR_OOM; }
    ora_moments(0, dims, NULL, f, rho, u);
    for (n = 0; n < N; ++n) {
        int64_t xp = shifted_node(dims, n, 1, 0, 0), xm = shifted_node(dims, n, -1, 0, 0);
        int64_t yp = shifted_node(dims, n, 0, 1, 0), ym = shifted_node(dims, n, 0, -1, 0);
        w[n] = 0.5 * (u[N + xp] - u[N + xm]) - 0.5 * (u[yp] - u[ym]);
        acc += u[n] * u[n] + u[N + n] * u[N + n];
    }
    *E = 0.5 * acc / (double)N;
    free(u);
    free(rho);
    return ORA_OK;
}

int ora_num_mlp(void) { return NMLP; }
int ora_num_theta(void) { return NTHETA; }

/* number of threads the node loops of ora_step use */
#ifdef _OPENMP
#include <omp.h>
int ora_num_threads(void) { return omp_get_max_threads(); }
#else
int ora_num_threads(void) { return 1; }
#endif
