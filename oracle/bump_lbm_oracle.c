/*
 * Reference oracle for the bump-function lattice Boltzmann scheme of
 * Afrasiabian & Denniston, "A Novel Velocity Discretization for Lattice
 * Boltzmann Method: Application to Compressible Flow" (arXiv 2501.00620).
 *
 * TEST INFRASTRUCTURE ONLY.  This is a plain, slow, double-precision CPU
 * restatement of the method, written to be checked against the paper by eye.
 * Only the test suite, the smoke check and the benchmark's CPU-baseline leg
 * may load it.  The product path (the CUDA library) shares no code, header,
 * table or helper with this file, and never calls it.
 *
 * Layout: array of sites, f[site*Q + i], b[site*NB + k].  Sites are numbered
 * x + nx*(y + ny*z).  The public entry points exchange structure-of-arrays
 * planes (field k of site s at k*N + s) so that they line up with the CUDA
 * library's boundary.
 *
 * Units: lattice units, dx = dt = c = 1.  tau is the paper's continuous
 * relaxation time (Sec. II.C), so the discrete relaxation factor is
 * omega = dt/(tau + dt/2) (Eq. 55).
 *
 * Order of one step (Sec. II.C, Eqs. 49-68), for the state (fbar, bbar) at t:
 *   A. per site: rho = sum fbar (Eq. 56); uncorrected momentum j0 = sum fbar e;
 *      u0 = j0/rho; the second-moment trace Ebar = sum fbar|e|^2 + rho tr bbar
 *      (Eq. 26 traced, barred variables); rho*b for the gradient from the
 *      explicit form of Eq. 68 with b^eq evaluated at the uncorrected u0.
 *   B. per site: F_beta = -d_alpha(rho b_alpha,beta) (Eq. 59),
 *      G_beta,gamma = -d_alpha(rho u_gamma b_alpha,beta + rho u_beta b_gamma,alpha)
 *      (Eq. 61, u taken as u0), isotropic central differences;
 *      corrected u = (j0 + F/2)/rho (Eq. 57); equilibria (Appendix A);
 *      forcing Phi_i with moments 0, F, G (Eqs. 58-61); SRT collision
 *      fbar* = fbar + omega(f^eq - fbar) + omega*tau*Phi (Eq. 55) and
 *      bbar* = bbar + dt*B = bbar + omega(b^eq - bbar) (Eqs. 63, 65).
 *   C. streaming: fbar_i(x, t+1) = fbar*_i(x - e_i) (Eq. 49) and the
 *      mass-weighted transport of bbar (Eq. 66).
 *
 * Readings where the paper is silent or ambiguous (each also listed in the
 * design notes of the repository):
 *   R1  D1Q3 and D2Q9 equilibria: obtained by collapsing the printed D3Q19
 *       equilibrium (Appendix A) onto the plane / line (sum the populations
 *       whose velocities project to the same lower-dimensional velocity).
 *   R2  Temperature: "isothermal" (paper: T is an input, P = rho T) uses T0
 *       everywhere; "thermal" takes T from the trace of the full second
 *       moment, T = (E - rho|u|^2)/(d rho), E = Ebar + tr(G)/2, so that the
 *       collision conserves E exactly.
 *   R3  tau is the continuous relaxation time: omega = 1/(tau + 1/2).
 *   R4  The weights in the bbar transport (Eq. 66) are the post-collision
 *       populations fbar*_i(x - e_i), i.e. exactly the numbers that stream
 *       into x, whose sum is rho(x, t+1).
 *   R5  Phi_i is the second-order Hermite projection with moments 0, F, G:
 *       Phi_i = w_i [ e_i.F / cs2 + (e_i e_i - cs2 I):G / (2 cs2^2) ].
 *   R6  Isotropic finite differences: d_alpha phi(x) = (1/cs2) sum_i w_i
 *       e_i,alpha phi(x + e_i), with the lattice weights w_i.
 *   R7  Start: at t = 0 every site emits its local equilibrium
 *       (fbar* = f^eq(rho0,u0), bbar* = b^eq(u0,T0)); the state at t = 0 is
 *       what streams in.
 *   R8  Fixed-state boundary (x only; y, z stay periodic): sites outside
 *       [0, nx) are frozen equilibrium reservoirs carrying the initial state of
 *       the edge site of their row.  They emit f^eq / b^eq of that state and
 *       present rho*b = rho b^eq and u0 = u to the gradient stencil.
 *   R9  Walls (Sec. III.A uses half-step bounce-back walls [Ladd 1994]): two
 *       stationary walls normal to the last axis (y in 2D, z in 3D), half a
 *       site outside the lattice, at -1/2 and n - 1/2; the other axes stay
 *       periodic.  A population whose source x - e_i lies beyond a wall is the
 *       one the site itself emitted in the opposite direction, fbar*_-i(x),
 *       and it carries that site's bbar*(x) in the transport of Eq. 66.  The
 *       gradient stencil sees, one site beyond a wall, the image of the fluid
 *       site facing it across the wall: the same rho*b and the reversed u0
 *       (bounce-back reverses velocities and leaves the variance unchanged).
 *   R12 Moving walls (Sec. III.D's Couette flow): a wall may move along
 *       itself with velocity u_w (lower wall u_lo, upper wall u_hi).  A
 *       population bounced at it gains the momentum of the wall,
 *       fbar_i(x, t+1) = fbar*_-i(x, t) + 6 w_i rho(x, t) e_i.u_w, with
 *       rho(x, t) the sum of the site's own emissions (the odd part of the
 *       equilibrium is exactly 6 w_i rho e_i.u, so a site moving with the
 *       wall at equilibrium is reproduced); its bbar is unchanged.  The
 *       gradient stencil's image velocity is reflected about the wall's,
 *       2 u_w - u0.
 *   R13 MRT collision (Appendix B; the paper itself runs SRT): D3Q19, in
 *       the moment basis m of Table M.  The appendix leaves w_i and N^a
 *       undefined: w_i are the lattice weights and N^a = 1 / sum_i w_i
 *       (m^a_i)^2 -- the rows of Table M are orthogonal under the weighted
 *       sum, so f_i = w_i sum_a m^a_i N^a M^a inverts M^a = sum_i m^a_i f_i.
 *       Each moment relaxes at its own rate with the forcing weighted as in
 *       the SRT step: M*^a = M^a + s_a (M^a_eq - M^a) + (1 - s_a/2) Phi^a,
 *       Phi^a = sum_i m^a_i Phi_i; s_a = omega for the conserved and the
 *       second-order rows (so eta = rho T tau and the energy of the thermal
 *       mode are those of the SRT step), s3 for the third-order rows 10-15,
 *       s4 for the fourth-order rows 16-18.  With s3 = s4 = omega it is the
 *       SRT step (1 - omega/2 = omega tau).  bbar keeps the single rate.
 *   R10 Body force (Sec. III.A drives Poiseuille flow by a uniform
 *       acceleration a): the force density rho a joins the gradient force,
 *       F -> F + rho a, and its second-moment source joins G,
 *       G_bc -> G_bc + rho (u_b a_c + u_c a_b) with the corrected velocity
 *       u = (j0 + F/2)/rho of Eq. 57, so that the forcing projection (R5)
 *       carries both and, in a uniform flow, the work of the force goes into
 *       kinetic energy alone (the thermal T stays constant).
 *
 * Standard-lattice comparator (model 1; periodic, or walls): the textbook BGK
 * scheme with the second-order Hermite equilibrium of Eq. 4 written in
 * lattice units, f^eq_i = w_i rho [1 + e.u/cs2 + (u u + (T0 - cs2) I) :
 * (e e - cs2 I) / (2 cs2^2)], collided with the same omega = 1/(tau + 1/2)
 * and streamed like the populations of the bump scheme; no variance, no
 * gradient correction.  A body force enters by the textbook second-order
 * forcing (the projection R5 with F = rho a, G = rho (u a + a u)).  Its moments through second order are rho, rho u and
 * rho (T0 I + u u); its third moment is fixed by the lattice (Sec. I), which
 * is what the bump scheme corrects.
 *
 * Weights w_i = f^eq_i(rho=1, u=0), cs2 = c^2/3 = 1/3.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define QMAX 19
#define NBMAX 6

typedef struct {
    int d, Q, nb;
    int e[QMAX][3];
    int opp[QMAX];             /* index of -e_i */
    double w[QMAX];
} orc_lattice;

typedef struct {
    orc_lattice L;
    int nx, ny, nz;
    long N;
    double tau, T0, omega;
    int thermal, bc;           /* bc: 0 periodic, 1 fixed-state in x, 2 walls (R9) */
    int model;                 /* 0 bump-function scheme, 1 standard comparator */
    int mrt;                   /* 1: MRT collision in the basis of Table M (R13) */
    double srate[QMAX];        /* its per-moment relaxation rates */
    double acc[3];             /* uniform body-force acceleration (R10) */
    double uw[2][3];           /* wall velocities (R12): [0] lower, [1] upper */
    long nstep;
    /* state at time t (pre-collision, post-stream) */
    double *f, *b;
    /* emitted (post-collision) state of the last collision, or of the start */
    double *fs, *bs;
    /* phase A per-site quantities */
    double *rho, *j0, *Ebar, *u0, *rb;
    /* phase B per-site quantities kept for moments / diagnostics */
    double *F, *G;
    /* fixed-state reservoirs: [side][row]  (side 0: x < 0, side 1: x >= nx) */
    long nrow;
    double *g_fs, *g_bs, *g_rho, *g_u, *g_rb;
} orc_sim;

/* ---------------------------------------------------------------------- */
/* Velocity sets.  D3Q19 ordering is the column order of the population-to-
 * moment matrix of Appendix B (its rows 2-4 are e_x, e_y, e_z).  D2Q9 and
 * D1Q3 orders follow the same pattern: rest, +x, +y, -x, -y, then diagonals
 * (++, +-, -+, --).                                                       */

static const int E1[3][3] = {{0, 0, 0}, {1, 0, 0}, {-1, 0, 0}};
static const int E2[9][3] = {{0, 0, 0}, {1, 0, 0},  {0, 1, 0},
                             {-1, 0, 0}, {0, -1, 0}, {1, 1, 0},
                             {1, -1, 0}, {-1, 1, 0}, {-1, -1, 0}};
static const int E3[19][3] = {
    {0, 0, 0},  {1, 0, 0},  {0, 1, 0},   {-1, 0, 0},  {0, -1, 0},
    {0, 0, 1},  {0, 0, -1}, {1, 1, 0},   {1, -1, 0},  {-1, 1, 0},
    {-1, -1, 0}, {1, 0, 1}, {1, 0, -1},  {-1, 0, 1},  {-1, 0, -1},
    {0, 1, 1},  {0, 1, -1}, {0, -1, 1},  {0, -1, -1}};

/* Table M (Appendix B): the D3Q19 population-to-moment matrix with c = 1,
 * row a = moment a, column i = population i in the order above.  Each row is
 * written as integers over a common denominator (TM_DEN).                   */
static const int TM_NUM[19][19] = {
    {1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1},
    {0, 1, 0, -1, 0, 0, 0, 1, 1, -1, -1, 1, 1, -1, -1, 0, 0, 0, 0},
    {0, 0, 1, 0, -1, 0, 0, 1, -1, 1, -1, 0, 0, 0, 0, 1, 1, -1, -1},
    {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1},
    {-1, 2, -1, 2, -1, -1, -1, 2, 2, 2, 2, 2, 2, 2, 2, -1, -1, -1, -1},
    {-1, -1, 2, -1, 2, -1, -1, 2, 2, 2, 2, -1, -1, -1, -1, 2, 2, 2, 2},
    {-1, -1, -1, -1, -1, 2, 2, -1, -1, -1, -1, 2, 2, 2, 2, 2, 2, 2, 2},
    {0, 0, 0, 0, 0, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 0, 0, 0, 0},
    {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0},
    {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 1, -1, -1, 1},
    {0, -2, 0, 2, 0, 0, 0, 1, 1, -1, -1, 1, 1, -1, -1, 0, 0, 0, 0},
    {0, 0, -2, 0, 2, 0, 0, 1, -1, 1, -1, 0, 0, 0, 0, 1, 1, -1, -1},
    {0, 0, 0, 0, 0, -2, 2, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1},
    {0, 0, 0, 0, 0, 0, 0, 1, 1, -1, -1, -1, -1, 1, 1, 0, 0, 0, 0},
    {0, 0, 0, 0, 0, 0, 0, 1, -1, 1, -1, 0, 0, 0, 0, -1, -1, 1, 1},
    {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 1, -1, 1, -1, -1, 1, -1, 1},
    {0, 1, 1, 1, 1, -2, -2, -2, -2, -2, -2, 1, 1, 1, 1, 1, 1, 1, 1},
    {0, 1, -1, 1, -1, 0, 0, 0, 0, 0, 0, -1, -1, -1, -1, 1, 1, 1, 1},
    {1, -2, -2, -2, -2, -2, -2, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1}};
static const int TM_DEN[19] = {1, 1, 1, 1, 3, 3, 3, 1, 1, 1, 3, 3, 3, 1, 1, 1, 2, 2, 6};

static double tm(int a, int i) { return (double)TM_NUM[a][i] / (double)TM_DEN[a]; }

/* MRT collision of one site (R13): moments of f, f^eq and Phi, relaxation
 * per moment, back to populations.                                        */
static void mrt_collide(const orc_sim *s, const double *f, const double *fe, const double *phi, double *fs)
{
    const orc_lattice *L = &s->L;
    double Ms[19];
    for (int a = 0; a < 19; ++a) {
        double M = 0.0, Me = 0.0, P = 0.0;
        for (int i = 0; i < 19; ++i) {
            M += tm(a, i) * f[i];
            Me += tm(a, i) * fe[i];
            P += tm(a, i) * phi[i];
        }
        Ms[a] = M + s->srate[a] * (Me - M) + (1.0 - 0.5 * s->srate[a]) * P;
    }
    for (int i = 0; i < 19; ++i) {
        double acc = 0.0;
        for (int a = 0; a < 19; ++a) {
            double Na = 0.0;                       /* 1 / sum_k w_k m_ak^2 */
            for (int k = 0; k < 19; ++k) Na += L->w[k] * tm(a, k) * tm(a, k);
            acc += tm(a, i) * Ms[a] / Na;
        }
        fs[i] = L->w[i] * acc;
    }
}

/* symmetric tensor component order: 1D (xx); 2D (xx, yy, xy);
 * 3D (xx, yy, zz, xy, xz, yz) */
static int comp_index(int d, int a, int b)
{
    if (a == b) return a;
    if (a > b) { int t = a; a = b; b = t; }
    if (d == 2) return 2;                 /* xy */
    if (a == 0 && b == 1) return 3;       /* xy */
    if (a == 0 && b == 2) return 4;       /* xz */
    return 5;                             /* yz */
}

/* ---------------------------------------------------------------------- */
/* Equilibria (Appendix A, and reading R1 for d = 1, 2).  c = 1.           */

static void feq_3d(double rho, const double *u, double *f)
{
    double ux = u[0], uy = u[1], uz = u[2];
    double x2 = ux * ux, y2 = uy * uy, z2 = uz * uz;
    f[0] = rho * (3.0 - 2.0 * (x2 + y2 + z2) - 6.0 * ((y2 + z2) * x2 + y2 * z2)) / 9.0;
    f[1] = rho * (1.0 + 3.0 * ux + 2.0 * (x2 - y2 - z2) + 6.0 * x2 * (y2 + z2)) / 18.0;
    f[2] = rho * (1.0 + 3.0 * uy - 2.0 * (x2 - y2 + z2) + 6.0 * y2 * (x2 + z2)) / 18.0;
    f[3] = rho * (1.0 - 3.0 * ux + 2.0 * (x2 - y2 - z2) + 6.0 * x2 * (y2 + z2)) / 18.0;
    f[4] = rho * (1.0 - 3.0 * uy - 2.0 * (x2 - y2 + z2) + 6.0 * y2 * (x2 + z2)) / 18.0;
    f[5] = rho * (1.0 + 3.0 * uz - 2.0 * (x2 + y2 - z2) + 6.0 * (x2 + y2) * z2) / 18.0;
    f[6] = rho * (1.0 - 3.0 * uz - 2.0 * (x2 + y2 - z2) + 6.0 * (x2 + y2) * z2) / 18.0;
    f[7] = rho * (1.0 + 3.0 * (ux + uy) + 2.0 * (x2 + 3.0 * uy * ux + y2) - 6.0 * x2 * y2) / 36.0;
    f[8] = rho * (1.0 + 3.0 * (ux - uy) + 2.0 * (x2 - 3.0 * uy * ux + y2) - 6.0 * x2 * y2) / 36.0;
    f[9] = rho * (1.0 - 3.0 * (ux - uy) + 2.0 * (x2 - 3.0 * uy * ux + y2) - 6.0 * x2 * y2) / 36.0;
    f[10] = rho * (1.0 - 3.0 * (ux + uy) + 2.0 * (x2 + 3.0 * uy * ux + y2) - 6.0 * x2 * y2) / 36.0;
    f[11] = rho * (1.0 + 3.0 * (ux + uz) + 2.0 * (x2 + 3.0 * uz * ux + z2) - 6.0 * x2 * z2) / 36.0;
    f[12] = rho * (1.0 + 3.0 * (ux - uz) + 2.0 * (x2 - 3.0 * uz * ux + z2) - 6.0 * x2 * z2) / 36.0;
    f[13] = rho * (1.0 - 3.0 * (ux - uz) + 2.0 * (x2 - 3.0 * uz * ux + z2) - 6.0 * x2 * z2) / 36.0;
    f[14] = rho * (1.0 - 3.0 * (ux + uz) + 2.0 * (x2 + 3.0 * uz * ux + z2) - 6.0 * x2 * z2) / 36.0;
    f[15] = rho * (1.0 + 3.0 * (uy + uz) + 2.0 * (y2 + 3.0 * uz * uy + z2) - 6.0 * y2 * z2) / 36.0;
    f[16] = rho * (1.0 + 3.0 * (uy - uz) + 2.0 * (y2 - 3.0 * uz * uy + z2) - 6.0 * y2 * z2) / 36.0;
    f[17] = rho * (1.0 - 3.0 * (uy - uz) + 2.0 * (y2 - 3.0 * uz * uy + z2) - 6.0 * y2 * z2) / 36.0;
    f[18] = rho * (1.0 - 3.0 * (uy + uz) + 2.0 * (y2 + 3.0 * uz * uy + z2) - 6.0 * y2 * z2) / 36.0;
}

/* D2Q9: Appendix A with u_z = 0, populations summed over e_z (reading R1). */
static void feq_2d(double rho, const double *u, double *f)
{
    double ux = u[0], uy = u[1];
    double x2 = ux * ux, y2 = uy * uy;
    f[0] = 2.0 * rho * (2.0 - 2.0 * (x2 + y2) - 3.0 * x2 * y2) / 9.0;
    f[1] = rho * (1.0 + 3.0 * ux + 2.0 * x2 - y2 + 3.0 * x2 * y2) / 9.0;
    f[2] = rho * (1.0 + 3.0 * uy + 2.0 * y2 - x2 + 3.0 * x2 * y2) / 9.0;
    f[3] = rho * (1.0 - 3.0 * ux + 2.0 * x2 - y2 + 3.0 * x2 * y2) / 9.0;
    f[4] = rho * (1.0 - 3.0 * uy + 2.0 * y2 - x2 + 3.0 * x2 * y2) / 9.0;
    f[5] = rho * (1.0 + 3.0 * (ux + uy) + 2.0 * (x2 + 3.0 * ux * uy + y2) - 6.0 * x2 * y2) / 36.0;
    f[6] = rho * (1.0 + 3.0 * (ux - uy) + 2.0 * (x2 - 3.0 * ux * uy + y2) - 6.0 * x2 * y2) / 36.0;
    f[7] = rho * (1.0 - 3.0 * (ux - uy) + 2.0 * (x2 - 3.0 * ux * uy + y2) - 6.0 * x2 * y2) / 36.0;
    f[8] = rho * (1.0 - 3.0 * (ux + uy) + 2.0 * (x2 + 3.0 * ux * uy + y2) - 6.0 * x2 * y2) / 36.0;
}

/* D1Q3: the D2Q9 form with u_y = 0, summed over e_y (reading R1). */
static void feq_1d(double rho, const double *u, double *f)
{
    double ux = u[0];
    f[0] = 2.0 * rho * (1.0 - ux * ux) / 3.0;
    f[1] = rho * (1.0 + ux) * (1.0 + 2.0 * ux) / 6.0;
    f[2] = rho * (1.0 - ux) * (1.0 - 2.0 * ux) / 6.0;
}

static void feq(int d, double rho, const double *u, double *f)
{
    if (d == 3) feq_3d(rho, u, f);
    else if (d == 2) feq_2d(rho, u, f);
    else feq_1d(rho, u, f);
}

/* b^eq_ab = T delta_ab + (u_a u_b - c^2 delta_ab)/3   (Eq. 36 with
 * P = rho T delta, written componentwise in Appendix A). */
static void beq(int d, const double *u, double T, double *bq)
{
    for (int a = 0; a < d; ++a)
        for (int c = a; c < d; ++c) {
            double v = u[a] * u[c] / 3.0;
            if (a == c) v += T - 1.0 / 3.0;
            bq[comp_index(d, a, c)] = v;
        }
}

/* Forcing projection (reading R5): moments 0, F and G of Eqs. 58-61. */
static void forcing(const orc_lattice *L, const double *F, const double *G, double *phi)
{
    const double cs2 = 1.0 / 3.0;
    int d = L->d;
    for (int i = 0; i < L->Q; ++i) {
        double eF = 0.0, eGe = 0.0, trG = 0.0;
        for (int a = 0; a < d; ++a) {
            eF += L->e[i][a] * F[a];
            trG += G[comp_index(d, a, a)];
            for (int c = 0; c < d; ++c)
                eGe += L->e[i][a] * L->e[i][c] * G[comp_index(d, a, c)];
        }
        phi[i] = L->w[i] * (eF / cs2 + (eGe - cs2 * trG) / (2.0 * cs2 * cs2));
    }
}

/* Standard-lattice equilibrium (Eq. 4 in lattice units, cs2 = 1/3).       */
static void std_feq(const orc_lattice *L, double rho, const double *u, double T, double *f)
{
    int d = L->d;
    double uu = 0.0;
    for (int a = 0; a < d; ++a) uu += u[a] * u[a];
    for (int i = 0; i < L->Q; ++i) {
        double eu = 0.0, ee = 0.0;
        for (int a = 0; a < d; ++a) {
            eu += L->e[i][a] * u[a];
            ee += (double)(L->e[i][a] * L->e[i][a]);
        }
        /* (u u + (T - cs2) I) : (e e - cs2 I) = (e.u)^2 - cs2 |u|^2 + (T - cs2)(|e|^2 - d cs2) */
        double second = eu * eu - uu / 3.0 + (T - 1.0 / 3.0) * (ee - d / 3.0);
        f[i] = L->w[i] * rho * (1.0 + 3.0 * eu + 4.5 * second);
    }
}

static void lattice_init(orc_lattice *L, int d)
{
    const int(*E)[3] = d == 3 ? E3 : (d == 2 ? E2 : E1);
    L->d = d;
    L->Q = d == 3 ? 19 : (d == 2 ? 9 : 3);
    L->nb = d == 3 ? 6 : (d == 2 ? 3 : 1);
    double zero[3] = {0.0, 0.0, 0.0};
    double w[QMAX];
    feq(d, 1.0, zero, w);               /* w_i = f^eq_i(1, 0) */
    for (int i = 0; i < L->Q; ++i) {
        for (int a = 0; a < 3; ++a) L->e[i][a] = E[i][a];
        L->w[i] = w[i];
    }
    for (int i = 0; i < L->Q; ++i)
        for (int j = 0; j < L->Q; ++j)
            if (E[j][0] == -E[i][0] && E[j][1] == -E[i][1] && E[j][2] == -E[i][2]) L->opp[i] = j;
}

/* ---------------------------------------------------------------------- */
/* Neighbours.  Returns the site index of (x,y,z)+s, or, for a fixed-state
 * boundary, -1 - (side*nrow + row) for a reservoir site.                   */

static long neighbour(const orc_sim *s, int x, int y, int z, int sx, int sy, int sz)
{
    int X = x + sx, Y = y + sy, Z = z + sz;
    if (s->bc == 2) {           /* walls: callers resolve the wall axis first */
        X = ((X % s->nx) + s->nx) % s->nx;
        if (s->L.d == 3) Y = ((Y % s->ny) + s->ny) % s->ny;
        return (long)X + (long)s->nx * ((long)Y + (long)s->ny * Z);
    }
    Y = ((Y % s->ny) + s->ny) % s->ny;
    Z = ((Z % s->nz) + s->nz) % s->nz;
    if (s->bc == 1 && (X < 0 || X >= s->nx)) {
        long row = (long)Y + (long)s->ny * Z;
        int side = X < 0 ? 0 : 1;
        return -1 - ((long)side * s->nrow + row);
    }
    X = ((X % s->nx) + s->nx) % s->nx;
    return (long)X + (long)s->nx * ((long)Y + (long)s->ny * Z);
}

/* Coordinate along the wall axis (R9) of (x,y,z) and its extent.          */
static int wall_coord(const orc_sim *s, int y, int z) { return s->L.d == 3 ? z : y; }
static int wall_extent(const orc_sim *s) { return s->L.d == 3 ? s->nz : s->ny; }

/* Gradient-stencil neighbour (x,y,z) + e under the walls of R9: the fluid
 * site facing it across the wall.  *wall = -1 for a fluid neighbour, else
 * the wall crossed (0 lower, 1 upper), whose image velocity is
 * 2 u_w - u0 (R9, R12).                                                    */
static long grad_neighbour(const orc_sim *s, int x, int y, int z, const int *e, int *wall)
{
    *wall = -1;
    if (s->bc != 2) return neighbour(s, x, y, z, e[0], e[1], e[2]);
    int X = x + e[0], Y = y + e[1], Z = z + e[2];
    int w = wall_coord(s, Y, Z), n = wall_extent(s);
    if (w < 0 || w >= n) {
        int m = w < 0 ? -1 - w : 2 * n - 1 - w;      /* mirror across the wall */
        if (s->L.d == 3) Z = m; else Y = m;
        *wall = w < 0 ? 0 : 1;
    }
    return neighbour(s, X, Y, Z, 0, 0, 0);
}


static void site_coords(const orc_sim *s, long n, int *x, int *y, int *z)
{
    *x = (int)(n % s->nx);
    *y = (int)((n / s->nx) % s->ny);
    *z = (int)(n / ((long)s->nx * s->ny));
}

/* emitted populations / bbar / phase-A fields at a site or reservoir */
static const double *fs_at(const orc_sim *s, long k) { return k >= 0 ? s->fs + k * s->L.Q : s->g_fs + (-1 - k) * s->L.Q; }
static const double *bs_at(const orc_sim *s, long k) { return k >= 0 ? s->bs + k * s->L.nb : s->g_bs + (-1 - k) * s->L.nb; }
static const double *u0_at(const orc_sim *s, long k) { return k >= 0 ? s->u0 + k * 3 : s->g_u + (-1 - k) * 3; }
static const double *rb_at(const orc_sim *s, long k) { return k >= 0 ? s->rb + k * s->L.nb : s->g_rb + (-1 - k) * s->L.nb; }

/* u0 seen by the gradient stencil at neighbour m across `wall` (or not).   */
static void image_u0(const orc_sim *s, long m, int wall, double *u)
{
    const double *u0 = u0_at(s, m);
    for (int a = 0; a < 3; ++a) u[a] = wall < 0 ? u0[a] : 2.0 * s->uw[wall][a] - u0[a];
}

/* ---------------------------------------------------------------------- */
/* Phase A: uncorrected moments and rho*b for the gradient (Eqs. 56-57, 68) */

static void phase_a(orc_sim *s)
{
    const orc_lattice *L = &s->L;
    int d = L->d, Q = L->Q, nb = L->nb;
    long n;
#pragma omp parallel for schedule(static)
    for (n = 0; n < s->N; ++n) {
        const double *f = s->f + n * Q;
        const double *b = s->b + n * nb;
        double rho = 0.0, j[3] = {0.0, 0.0, 0.0}, e2 = 0.0;
        for (int i = 0; i < Q; ++i) {
            rho += f[i];
            for (int a = 0; a < d; ++a) j[a] += f[i] * L->e[i][a];
            double ee = 0.0;
            for (int a = 0; a < d; ++a) ee += (double)(L->e[i][a] * L->e[i][a]);
            e2 += f[i] * ee;
        }
        double trb = 0.0;
        for (int a = 0; a < d; ++a) trb += b[comp_index(d, a, a)];
        double Ebar = e2 + rho * trb;
        double u0[3] = {0.0, 0.0, 0.0}, uu = 0.0;
        for (int a = 0; a < d; ++a) { u0[a] = j[a] / rho; uu += u0[a] * u0[a]; }
        double Tunc = s->thermal ? (Ebar - rho * uu) / (d * rho) : s->T0;
        double bq[NBMAX];
        beq(d, u0, Tunc, bq);
        s->rho[n] = rho;
        s->Ebar[n] = Ebar;
        for (int a = 0; a < 3; ++a) { s->j0[n * 3 + a] = j[a]; s->u0[n * 3 + a] = u0[a]; }
        for (int k = 0; k < nb; ++k)
            s->rb[n * nb + k] = rho * b[k] - 0.5 * s->omega * (rho * b[k] - rho * bq[k]);
    }
}

/* Isotropic central difference (reading R6) of component k of rho*b, or of
 * H_abc = u0_c rb_ab + u0_b rb_ca, taken along direction a, at site n.     */
static double grad_rb(const orc_sim *s, int x, int y, int z, int a, int k)
{
    const orc_lattice *L = &s->L;
    double acc = 0.0;
    for (int i = 1; i < L->Q; ++i) {
        if (L->e[i][a] == 0) continue;
        int wall;
        long m = grad_neighbour(s, x, y, z, L->e[i], &wall);
        acc += L->w[i] * L->e[i][a] * rb_at(s, m)[k];
    }
    return 3.0 * acc;
}

static double grad_H(const orc_sim *s, int x, int y, int z, int a, int bb, int c)
{
    const orc_lattice *L = &s->L;
    int d = L->d;
    double acc = 0.0;
    for (int i = 1; i < L->Q; ++i) {
        if (L->e[i][a] == 0) continue;
        int wall;
        double u[3];
        long m = grad_neighbour(s, x, y, z, L->e[i], &wall);
        image_u0(s, m, wall, u);
        const double *r = rb_at(s, m);
        double H = u[c] * r[comp_index(d, a, bb)] + u[bb] * r[comp_index(d, c, a)];
        acc += L->w[i] * L->e[i][a] * H;
    }
    return 3.0 * acc;
}

/* Phase B (first half): F, G (Eqs. 59, 61) and the corrected u, T.          */
static void corrected_moments(const orc_sim *s, long n, double *F, double *G,
                              double *u, double *T)
{
    int d = s->L.d, nb = s->L.nb;
    int x, y, z;
    site_coords(s, n, &x, &y, &z);
    for (int bb = 0; bb < d; ++bb) {
        double acc = 0.0;
        for (int a = 0; a < d; ++a) acc += grad_rb(s, x, y, z, a, comp_index(d, a, bb));
        F[bb] = -acc;
    }
    for (int k = 0; k < nb; ++k) G[k] = 0.0;
    for (int bb = 0; bb < d; ++bb)
        for (int c = bb; c < d; ++c) {
            double acc = 0.0;
            for (int a = 0; a < d; ++a) acc += grad_H(s, x, y, z, a, bb, c);
            G[comp_index(d, bb, c)] = -acc;
        }
    double rho = s->rho[n], uu = 0.0, trG = 0.0;
    /* body force (R10): F + rho a, then G + rho (u a + a u) with the
     * corrected momentum rho u = j0 + F/2 of Eq. 57 */
    double ru[3] = {0.0, 0.0, 0.0};
    for (int bb = 0; bb < d; ++bb) F[bb] += rho * s->acc[bb];
    for (int bb = 0; bb < d; ++bb) ru[bb] = s->j0[n * 3 + bb] + 0.5 * F[bb];
    for (int bb = 0; bb < d; ++bb)
        for (int c = bb; c < d; ++c)
            G[comp_index(d, bb, c)] += ru[bb] * s->acc[c] + ru[c] * s->acc[bb];
    for (int a = 0; a < 3; ++a) u[a] = 0.0;
    for (int a = 0; a < d; ++a) {
        u[a] = (s->j0[n * 3 + a] + 0.5 * F[a]) / rho;     /* Eq. 57 */
        uu += u[a] * u[a];
        trG += G[comp_index(d, a, a)];
    }
    *T = (s->Ebar[n] + 0.5 * trG - rho * uu) / (d * rho);
}

/* Phase B (second half): equilibria, forcing and the SRT collision.         */
static void phase_b(orc_sim *s)
{
    const orc_lattice *L = &s->L;
    int d = L->d, Q = L->Q, nb = L->nb;
    double om = s->omega, tau = s->tau;
    long n;
#pragma omp parallel for schedule(static)
    for (n = 0; n < s->N; ++n) {
        double F[3] = {0, 0, 0}, G[NBMAX], u[3], Tm, fe[QMAX], bq[NBMAX], phi[QMAX];
        corrected_moments(s, n, F, G, u, &Tm);
        double T = s->thermal ? Tm : s->T0;
        feq(d, s->rho[n], u, fe);
        beq(d, u, T, bq);
        forcing(L, F, G, phi);
        for (int a = 0; a < 3; ++a) s->F[n * 3 + a] = F[a];
        for (int k = 0; k < nb; ++k) s->G[n * nb + k] = G[k];
        const double *f = s->f + n * Q, *b = s->b + n * nb;
        double *fs = s->fs + n * Q, *bs = s->bs + n * nb;
        if (s->mrt)                                        /* R13 */
            mrt_collide(s, f, fe, phi, fs);
        else
            for (int i = 0; i < Q; ++i)                    /* Eq. 55 */
                fs[i] = f[i] + om * (fe[i] - f[i]) + om * tau * phi[i];
        for (int k = 0; k < nb; ++k)                       /* Eqs. 63, 65 */
            bs[k] = b[k] + om * (bq[k] - b[k]);
    }
}

/* Standard comparator: moments and BGK collision with the equilibrium of
 * Eq. 4; fs = f + omega (f^eq - f).                                        */
static void std_moments(const orc_sim *s, long n, double *rho, double *j, double *E)
{
    const orc_lattice *L = &s->L;
    const double *f = s->f + n * L->Q;
    *rho = 0.0;
    *E = 0.0;
    for (int a = 0; a < 3; ++a) j[a] = 0.0;
    for (int i = 0; i < L->Q; ++i) {
        double ee = 0.0;
        *rho += f[i];
        for (int a = 0; a < L->d; ++a) {
            j[a] += f[i] * L->e[i][a];
            ee += (double)(L->e[i][a] * L->e[i][a]);
        }
        *E += f[i] * ee;
    }
}

static void std_collide(orc_sim *s)
{
    const orc_lattice *L = &s->L;
    int Q = L->Q, d = L->d;
    long n;
#pragma omp parallel for schedule(static)
    for (n = 0; n < s->N; ++n) {
        double rho, j[3], E, u[3] = {0.0, 0.0, 0.0}, fe[QMAX];
        double F[3] = {0.0, 0.0, 0.0}, G[NBMAX], phi[QMAX];
        std_moments(s, n, &rho, j, &E);
        /* body force: the textbook second-order (Guo-type) scheme, i.e. the
         * forcing projection R5 with F = rho a, G = rho (u a + a u) and the
         * half-force velocity, weighted by omega tau = 1 - omega/2 */
        for (int a = 0; a < d; ++a) {
            F[a] = rho * s->acc[a];
            u[a] = (j[a] + 0.5 * F[a]) / rho;
        }
        for (int a = 0; a < d; ++a)
            for (int c = a; c < d; ++c)
                G[comp_index(d, a, c)] = rho * (u[a] * s->acc[c] + u[c] * s->acc[a]);
        std_feq(L, rho, u, s->T0, fe);
        forcing(L, F, G, phi);
        const double *f = s->f + n * Q;
        double *fs = s->fs + n * Q;
        for (int i = 0; i < Q; ++i) fs[i] = f[i] + s->omega * (fe[i] - f[i]) + s->omega * s->tau * phi[i];
    }
}

/* Phase C: streaming of fbar (Eq. 49) and transport of bbar (Eq. 66, R4).   */
static void phase_c(orc_sim *s)
{
    const orc_lattice *L = &s->L;
    int Q = L->Q, nb = L->nb;
    long n;
#pragma omp parallel for schedule(static)
    for (n = 0; n < s->N; ++n) {
        int x, y, z;
        site_coords(s, n, &x, &y, &z);
        double rho1 = 0.0, rbb[NBMAX];
        for (int k = 0; k < nb; ++k) rbb[k] = 0.0;
        for (int i = 0; i < Q; ++i) {
            double fi;
            const double *bm;
            int w = wall_coord(s, y - L->e[i][1], z - L->e[i][2]);
            if (s->bc == 2 && (w < 0 || w >= wall_extent(s))) {
                /* half-way bounce-back (R9): the site's own opposite
                 * emission, plus the wall's momentum (R12) */
                const double *uw = s->uw[w < 0 ? 0 : 1];
                double eu = 0.0, rho0 = 0.0;
                for (int a = 0; a < L->d; ++a) eu += L->e[i][a] * uw[a];
                if (eu != 0.0)
                    for (int k = 0; k < Q; ++k) rho0 += s->fs[n * Q + k];
                fi = s->fs[n * Q + L->opp[i]] + 6.0 * L->w[i] * rho0 * eu;
                bm = s->bs + n * nb;
            } else {
                long m = neighbour(s, x, y, z, -L->e[i][0], -L->e[i][1], -L->e[i][2]);
                fi = fs_at(s, m)[i];
                bm = bs_at(s, m);
            }
            s->f[n * Q + i] = fi;
            rho1 += fi;
            for (int k = 0; k < nb; ++k) rbb[k] += fi * bm[k];
        }
        for (int k = 0; k < nb; ++k) s->b[n * nb + k] = rbb[k] / rho1;
    }
}

/* ---------------------------------------------------------------------- */
/* Public entry points (ctypes).                                           */

int orc_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

int orc_lattice_info(int d, int *Q, int *nb, int *e, double *w)
{
    if (d < 1 || d > 3) return -1;
    orc_lattice L;
    lattice_init(&L, d);
    *Q = L.Q;
    *nb = L.nb;
    if (e) for (int i = 0; i < L.Q; ++i) for (int a = 0; a < 3; ++a) e[i * 3 + a] = L.e[i][a];
    if (w) for (int i = 0; i < L.Q; ++i) w[i] = L.w[i];
    return 0;
}

void orc_feq(int d, double rho, const double *u, double *out) { double uu[3] = {0, 0, 0}; for (int a = 0; a < d; ++a) uu[a] = u[a]; feq(d, rho, uu, out); }
void orc_beq(int d, const double *u, double T, double *out) { beq(d, u, T, out); }
void orc_forcing(int d, const double *F, const double *G, double *out)
{
    orc_lattice L;
    lattice_init(&L, d);
    double FF[3] = {0, 0, 0};
    for (int a = 0; a < d; ++a) FF[a] = F[a];
    forcing(&L, FF, G, out);
}

void orc_destroy(void *h)
{
    orc_sim *s = (orc_sim *)h;
    if (!s) return;
    free(s->f); free(s->b); free(s->fs); free(s->bs);
    free(s->rho); free(s->j0); free(s->Ebar); free(s->u0); free(s->rb);
    free(s->F); free(s->G);
    free(s->g_fs); free(s->g_bs); free(s->g_rho); free(s->g_u); free(s->g_rb);
    free(s);
}

void *orc_create(int d, int nx, int ny, int nz, double tau, double T0, int thermal, int bc)
{
    if (d < 1 || d > 3 || nx < 1 || ny < 1 || nz < 1 || !(tau > 0) || !(T0 > 0)) return NULL;
    if ((d < 2 && ny != 1) || (d < 3 && nz != 1)) return NULL;
    if (bc < 0 || bc > 2 || (bc == 2 && d < 2)) return NULL;
    orc_sim *s = (orc_sim *)calloc(1, sizeof(orc_sim));
    lattice_init(&s->L, d);
    s->nx = nx; s->ny = ny; s->nz = nz;
    s->N = (long)nx * ny * nz;
    s->tau = tau; s->T0 = T0; s->omega = 1.0 / (tau + 0.5);
    s->thermal = thermal; s->bc = bc;
    s->nrow = (long)ny * nz;
    int Q = s->L.Q, nb = s->L.nb;
    long N = s->N;
    s->f = calloc(N * Q, sizeof(double)); s->fs = calloc(N * Q, sizeof(double));
    s->b = calloc(N * nb, sizeof(double)); s->bs = calloc(N * nb, sizeof(double));
    s->rho = calloc(N, sizeof(double)); s->Ebar = calloc(N, sizeof(double));
    s->j0 = calloc(N * 3, sizeof(double)); s->u0 = calloc(N * 3, sizeof(double));
    s->rb = calloc(N * nb, sizeof(double));
    s->F = calloc(N * 3, sizeof(double)); s->G = calloc(N * nb, sizeof(double));
    long R = 2 * s->nrow;
    s->g_fs = calloc(R * Q, sizeof(double)); s->g_bs = calloc(R * nb, sizeof(double));
    s->g_rho = calloc(R, sizeof(double)); s->g_u = calloc(R * 3, sizeof(double));
    s->g_rb = calloc(R * nb, sizeof(double));
    return s;
}

/* Start (reading R7): each site emits its local equilibrium, then streams. */
int orc_init(void *h, const double *rho, const double *u, const double *T)
{
    orc_sim *s = (orc_sim *)h;
    int d = s->L.d, Q = s->L.Q, nb = s->L.nb;
    long N = s->N;
    for (long n = 0; n < N; ++n) {
        double uu[3] = {0, 0, 0};
        for (int a = 0; a < d; ++a) uu[a] = u[a * N + n];
        if (!(rho[n] > 0) || !(T[n] > 0)) return -1;
        if (s->model == 1) {
            std_feq(&s->L, rho[n], uu, T[n], s->fs + n * Q);
            for (int k = 0; k < nb; ++k) s->bs[n * nb + k] = 0.0;
            continue;
        }
        feq(d, rho[n], uu, s->fs + n * Q);
        beq(d, uu, T[n], s->bs + n * nb);
    }
    /* reservoirs (reading R8): the initial state of the edge site of each row */
    for (int side = 0; side < 2; ++side)
        for (long row = 0; row < s->nrow; ++row) {
            long n = (long)(side ? s->nx - 1 : 0) + (long)s->nx * row;
            long g = side * s->nrow + row;
            double uu[3] = {0, 0, 0}, bq[NBMAX];
            for (int a = 0; a < d; ++a) uu[a] = u[a * N + n];
            feq(d, rho[n], uu, s->g_fs + g * Q);
            beq(d, uu, T[n], bq);
            s->g_rho[g] = rho[n];
            for (int a = 0; a < 3; ++a) s->g_u[g * 3 + a] = uu[a];
            for (int k = 0; k < nb; ++k) { s->g_bs[g * nb + k] = bq[k]; s->g_rb[g * nb + k] = rho[n] * bq[k]; }
        }
    phase_c(s);
    s->nstep = 0;
    return 0;
}

void orc_step(void *h, long nsteps)
{
    orc_sim *s = (orc_sim *)h;
    for (long t = 0; t < nsteps; ++t) {
        if (s->model == 1) {
            std_collide(s);
        } else {
            phase_a(s);
            phase_b(s);
        }
        phase_c(s);
        s->nstep++;
    }
}

long orc_nstep(void *h) { return ((orc_sim *)h)->nstep; }

/* Select the scheme before orc_init: 0 bump-function (default), 1 standard
 * comparator (periodic lattices or the walls of R9/R12, which bounce its
 * populations the same way).  Returns 0, or -1 if not allowed.            */
int orc_set_model(void *h, int model)
{
    orc_sim *s = (orc_sim *)h;
    if (model < 0 || model > 1 || (model == 1 && s->bc == 1)) return -1;
    s->model = model;
    return 0;
}

void orc_std_feq(int d, double rho, const double *u, double T, double *out)
{
    orc_lattice L;
    lattice_init(&L, d);
    double uu[3] = {0, 0, 0};
    for (int a = 0; a < d; ++a) uu[a] = u[a];
    std_feq(&L, rho, uu, T, out);
}

/* Wall velocities (R12): lower and upper, d components each, tangential
 * (the wall-normal component must be 0).  Returns 0, or -1 if not allowed. */
int orc_set_wall_velocity(void *h, const double *lo, const double *hi)
{
    orc_sim *s = (orc_sim *)h;
    int d = s->L.d, an = d - 1;
    if (s->bc != 2 || lo[an] != 0.0 || hi[an] != 0.0) return -1;
    for (int a = 0; a < 3; ++a) {
        s->uw[0][a] = a < d ? lo[a] : 0.0;
        s->uw[1][a] = a < d ? hi[a] : 0.0;
    }
    return 0;
}

/* MRT collision (R13), D3Q19 bump scheme only: rates s3 (third-order
 * moments) and s4 (fourth-order), each in (0, 2).  Returns 0 or -1.        */
int orc_set_mrt(void *h, double s3, double s4)
{
    orc_sim *s = (orc_sim *)h;
    if (s->L.d != 3 || s->model != 0 || !(s3 > 0 && s3 < 2) || !(s4 > 0 && s4 < 2)) return -1;
    for (int a = 0; a < 19; ++a) s->srate[a] = a < 10 ? s->omega : (a < 16 ? s3 : s4);
    s->mrt = 1;
    return 0;
}

/* Table M with c = 1, row-major (19 x 19).  Test hook.                     */
void orc_moment_matrix(double *out)
{
    for (int a = 0; a < 19; ++a)
        for (int i = 0; i < 19; ++i) out[a * 19 + i] = tm(a, i);
}

/* Uniform body-force acceleration (R10), d components.                    */
void orc_set_force(void *h, const double *a)
{
    orc_sim *s = (orc_sim *)h;
    for (int c = 0; c < 3; ++c) s->acc[c] = c < s->L.d ? a[c] : 0.0;
}

/* rho, corrected u (d planes) and the moment temperature at the current t */
void orc_moments(void *h, double *rho, double *u, double *T)
{
    orc_sim *s = (orc_sim *)h;
    int d = s->L.d;
    long N = s->N;
    long n;
    if (s->model == 1) {          /* rho, u = (j + rho a/2)/rho, T = (E - rho|u|^2)/(d rho) */
        for (n = 0; n < N; ++n) {
            double r, j[3], E, uu = 0.0;
            std_moments(s, n, &r, j, &E);
            for (int a = 0; a < d; ++a) {
                double ua = (j[a] + 0.5 * r * s->acc[a]) / r;
                if (u) u[a * N + n] = ua;
                uu += ua * ua;
            }
            if (rho) rho[n] = r;
            if (T) T[n] = (E - r * uu) / (d * r);
        }
        return;
    }
    phase_a(s);
#pragma omp parallel for schedule(static)
    for (n = 0; n < N; ++n) {
        double F[3] = {0, 0, 0}, G[NBMAX], uu[3], Tm;
        corrected_moments(s, n, F, G, uu, &Tm);
        if (rho) rho[n] = s->rho[n];
        if (u) for (int a = 0; a < d; ++a) u[a * N + n] = uu[a];
        if (T) T[n] = Tm;
    }
}

/* Global mass, momentum (d) and energy E = sum (Ebar + tr G / 2) in site
 * order: out[0] = M, out[1..d] = P, out[d+1] = E.                         */
void orc_diagnostics(void *h, double *out)
{
    orc_sim *s = (orc_sim *)h;
    int d = s->L.d, nb = s->L.nb;
    long N = s->N;
    if (s->model == 1) {          /* M, P = sum j, E = sum f|e|^2 */
        double M = 0.0, P[3] = {0, 0, 0}, E = 0.0;
        for (long n = 0; n < N; ++n) {
            double r, j[3], e2;
            std_moments(s, n, &r, j, &e2);
            M += r;
            for (int a = 0; a < d; ++a) P[a] += j[a] + 0.5 * r * s->acc[a];
            E += e2;
        }
        out[0] = M;
        for (int a = 0; a < d; ++a) out[1 + a] = P[a];
        out[1 + d] = E;
        return;
    }
    double *F = malloc(sizeof(double) * 3 * N), *G = malloc(sizeof(double) * nb * N);
    phase_a(s);
    long n;
#pragma omp parallel for schedule(static)
    for (n = 0; n < N; ++n) {
        double uu[3], Tm;
        corrected_moments(s, n, F + n * 3, G + n * nb, uu, &Tm);
    }
    double M = 0.0, P[3] = {0, 0, 0}, E = 0.0;
    for (n = 0; n < N; ++n) {
        M += s->rho[n];
        double trG = 0.0;
        for (int a = 0; a < d; ++a) {
            P[a] += s->j0[n * 3 + a] + 0.5 * F[n * 3 + a];
            trG += G[n * nb + comp_index(d, a, a)];
        }
        E += s->Ebar[n] + 0.5 * trG;
    }
    out[0] = M;
    for (int a = 0; a < d; ++a) out[1 + a] = P[a];
    out[1 + d] = E;
    free(F);
    free(G);
}

/* Emitted (post-collision) state of the last step: Q planes, nb planes.   */
void orc_get_emitted(void *h, double *f, double *b)
{
    orc_sim *s = (orc_sim *)h;
    int Q = s->L.Q, nb = s->L.nb;
    long N = s->N;
    for (long n = 0; n < N; ++n) {
        if (f) for (int i = 0; i < Q; ++i) f[i * N + n] = s->fs[n * Q + i];
        if (b) for (int k = 0; k < nb; ++k) b[k * N + n] = s->bs[n * nb + k];
    }
}

/* State at time t (pre-collision fbar, bbar): Q planes, nb planes.        */
void orc_get_state(void *h, double *f, double *b)
{
    orc_sim *s = (orc_sim *)h;
    int Q = s->L.Q, nb = s->L.nb;
    long N = s->N;
    for (long n = 0; n < N; ++n) {
        if (f) for (int i = 0; i < Q; ++i) f[i * N + n] = s->f[n * Q + i];
        if (b) for (int k = 0; k < nb; ++k) b[k * N + n] = s->b[n * nb + k];
    }
}

/* Isotropic gradient (reading R6) of a scalar field on a periodic lattice:
 * out[a*N + n] = (1/cs2) sum_i w_i e_ia phi(x_n + e_i).  Test hook.        */
void orc_gradient(int d, int nx, int ny, int nz, const double *phi, double *out)
{
    orc_sim *s = (orc_sim *)orc_create(d, nx, ny, nz, 1.0, 1.0, 0, 0);
    long N = s->N;
    for (long n = 0; n < N; ++n) {
        int x, y, z;
        site_coords(s, n, &x, &y, &z);
        for (int a = 0; a < d; ++a) {
            double acc = 0.0;
            for (int i = 1; i < s->L.Q; ++i) {
                if (s->L.e[i][a] == 0) continue;
                long m = neighbour(s, x, y, z, s->L.e[i][0], s->L.e[i][1], s->L.e[i][2]);
                acc += s->L.w[i] * s->L.e[i][a] * phi[m];
            }
            out[a * N + n] = 3.0 * acc;
        }
    }
    orc_destroy(s);
}

/* Replace the emitted state (Q planes, nb planes) and stream it, so that the
 * state at the current time is what these emissions deliver (Eqs. 49, 66).
 * Used to restart the oracle from a state produced elsewhere, e.g. a window
 * cut out of a larger periodic lattice: after one step, sites at distance
 * >= 2 from the window's edges are exact (the step reads the emitted state
 * up to two sites away: one for the pull, one for the gradient).          */
void orc_set_emitted(void *h, const double *f, const double *b)
{
    orc_sim *s = (orc_sim *)h;
    int Q = s->L.Q, nb = s->L.nb;
    long N = s->N;
    for (long n = 0; n < N; ++n) {
        for (int i = 0; i < Q; ++i) s->fs[n * Q + i] = f[i * N + n];
        for (int k = 0; k < nb; ++k) s->bs[n * nb + k] = b[k * N + n];
    }
    phase_c(s);
}
