/*
 * cmlbm_oracle.c -- plain, slow FP64 CPU oracle for the D3Q19 central-moment
 * lattice Boltzmann method of De Rosis & Coreixas, "Multiphysics flow
 * simulations using D3Q19 lattice Boltzmann methods based on central moments"
 * (arXiv:2010.01628).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or call
 * this file; only the test-suite, the smoke check and the benchmark's CPU
 * baseline use it.  It shares no code, header, table or constant with the CUDA
 * library: every lattice table below is typed in again from the paper.
 *
 * Two independent ways to do one collision are provided:
 *   - "dense" (Oracle-A): the definition.  Build the 19x19 matrix T(u) of
 *     Eq. (eq:matrix), compute k = T f, k_eq = T f_eq, R = T F_i and
 *     k* = (I-K)k + K k_eq + (I-K/2) R (Eq. eq:posColl0), then solve
 *     T f* = k* by Gaussian elimination with partial pivoting (Eq. system).
 *   - "closed" (Oracle-B): the paper's two-step reconstruction of App. C:
 *     post-collision CMs from the printed lists (Sec. II.B, App. E), raw
 *     moments r* = N^-1 k* (Eq. rawQ19) and populations f* = M^-1 r*
 *     (Eq. pdfQ19), with the misprints corrected as documented beside each
 *     line.
 *
 * Conventions (Sec. II): lattice units dx = dt = 1, c_s^2 = 1/3,
 * omega = 1/(nu/c_s^2 + 1/2).  All arithmetic is IEEE binary64; build with
 * -ffp-contract=off so no fused multiply-add changes the rounding.
 *
 * Time-step convention ("pull" order, a reading; the paper states collide then
 * stream): the stored state is the set of post-collision populations.  One
 * step gathers (streams) them into each node, applies the boundaries, takes
 * moments and collides.  The initial state is the equilibrium of the given
 * fields.  Reported fields are the moments of the gathered (post-stream)
 * populations, with +F/2 in the momentum (App. E, macroscopic variables).
 *
 * Shan-Chen multiphase (Sec. III.G, physics 3) takes two passes per step:
 * the pseudopotential psi = 1 - exp(-rho) of every node from its gathered
 * densities, then the single-phase collision with F = rho g + F_sc, where
 * F_sc = -G psi(x) sum_i w_i c_i psi(x + c_i).
 *
 * Populations are stored cell-major: f[cell*19 + i], cell = x + nx*(y + ny*z).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define Q 19
#define QM 7

/* Sec. II.A: the 19 lattice directions in the paper's order (the "swap"
 * ordering, opposite(i) = i +/- 9). */
static const int CX[Q] = {0, -1, 0, 0, -1, -1, -1, -1, 0, 0, 1, 0, 0, 1, 1, 1, 1, 0, 0};
static const int CY[Q] = {0, 0, -1, 0, -1, 1, 0, 0, -1, -1, 0, 1, 0, 1, -1, 0, 0, 1, 1};
static const int CZ[Q] = {0, 0, 0, -1, 0, 0, -1, 1, -1, 1, 0, 0, 1, 0, 0, 1, -1, 1, -1};

/* Sec. II.A weights: w0 = 1/3, ws = 1/18 (axis), wl = 1/36 (diagonal). */
static double weight(int i)
{
    int n2 = CX[i] * CX[i] + CY[i] * CY[i] + CZ[i] * CZ[i];
    if (n2 == 0) return 1.0 / 3.0;
    if (n2 == 1) return 1.0 / 18.0;
    return 1.0 / 36.0;
}

static int opposite(int i)
{
    if (i == 0) return 0;
    return i <= 9 ? i + 9 : i - 9;
}

static const double CS2 = 1.0 / 3.0;

int orc_lattice(int *cx, int *cy, int *cz, double *w)
{
    for (int i = 0; i < Q; i++) {
        cx[i] = CX[i];
        cy[i] = CY[i];
        cz[i] = CZ[i];
        w[i] = weight(i);
    }
    return Q;
}

/* ------------------------------------------------------------------------ */
/* Extended (fourth-order, D3Q19-pruned) equilibrium, Eq. (eq:EqQ19RM), written
 * out term by term in the paper's form. */
void orc_feq(double rho, double ux, double uy, double uz, double *f)
{
    double x2 = ux * ux, y2 = uy * uy, z2 = uz * uz;
    f[0] = rho / 3.0 * (1.0 - (x2 + y2 + z2) + 3.0 * (x2 * y2 + x2 * z2 + y2 * z2));
    f[1] = rho / 18.0 * (1.0 - 3.0 * ux + 3.0 * (x2 - y2 - z2) + 9.0 * (ux * y2 + ux * z2) - 9.0 * (x2 * y2 + x2 * z2));
    f[2] = rho / 18.0 * (1.0 - 3.0 * uy + 3.0 * (-x2 + y2 - z2) + 9.0 * (x2 * uy + uy * z2) - 9.0 * (x2 * y2 + y2 * z2));
    f[3] = rho / 18.0 * (1.0 - 3.0 * uz + 3.0 * (-x2 - y2 + z2) + 9.0 * (x2 * uz + y2 * uz) - 9.0 * (x2 * z2 + y2 * z2));
    f[4] = rho / 36.0 * (1.0 - 3.0 * (ux + uy) + 3.0 * (x2 + y2) + 9.0 * ux * uy - 9.0 * (x2 * uy + ux * y2) + 9.0 * x2 * y2);
    f[5] = rho / 36.0 * (1.0 + 3.0 * (-ux + uy) + 3.0 * (x2 + y2) - 9.0 * ux * uy + 9.0 * (x2 * uy - ux * y2) + 9.0 * x2 * y2);
    f[6] = rho / 36.0 * (1.0 - 3.0 * (ux + uz) + 3.0 * (x2 + z2) + 9.0 * ux * uz - 9.0 * (x2 * uz + ux * z2) + 9.0 * x2 * z2);
    f[7] = rho / 36.0 * (1.0 + 3.0 * (-ux + uz) + 3.0 * (x2 + z2) - 9.0 * ux * uz + 9.0 * (x2 * uz - ux * z2) + 9.0 * x2 * z2);
    f[8] = rho / 36.0 * (1.0 - 3.0 * (uy + uz) + 3.0 * (y2 + z2) + 9.0 * uy * uz - 9.0 * (y2 * uz + uy * z2) + 9.0 * y2 * z2);
    f[9] = rho / 36.0 * (1.0 + 3.0 * (-uy + uz) + 3.0 * (y2 + z2) - 9.0 * uy * uz + 9.0 * (y2 * uz - uy * z2) + 9.0 * y2 * z2);
    f[10] = rho / 18.0 * (1.0 + 3.0 * ux + 3.0 * (x2 - y2 - z2) - 9.0 * (ux * y2 + ux * z2) - 9.0 * (x2 * y2 + x2 * z2));
    f[11] = rho / 18.0 * (1.0 + 3.0 * uy + 3.0 * (-x2 + y2 - z2) - 9.0 * (x2 * uy + uy * z2) - 9.0 * (x2 * y2 + y2 * z2));
    f[12] = rho / 18.0 * (1.0 + 3.0 * uz + 3.0 * (-x2 - y2 + z2) - 9.0 * (x2 * uz + y2 * uz) - 9.0 * (x2 * z2 + y2 * z2));
    f[13] = rho / 36.0 * (1.0 + 3.0 * (ux + uy) + 3.0 * (x2 + y2) + 9.0 * ux * uy + 9.0 * (x2 * uy + ux * y2) + 9.0 * x2 * y2);
    f[14] = rho / 36.0 * (1.0 + 3.0 * (ux - uy) + 3.0 * (x2 + y2) - 9.0 * ux * uy + 9.0 * (-x2 * uy + ux * y2) + 9.0 * x2 * y2);
    f[15] = rho / 36.0 * (1.0 + 3.0 * (ux + uz) + 3.0 * (x2 + z2) + 9.0 * ux * uz + 9.0 * (x2 * uz + ux * z2) + 9.0 * x2 * z2);
    f[16] = rho / 36.0 * (1.0 + 3.0 * (ux - uz) + 3.0 * (x2 + z2) - 9.0 * ux * uz + 9.0 * (-x2 * uz + ux * z2) + 9.0 * x2 * z2);
    f[17] = rho / 36.0 * (1.0 + 3.0 * (uy + uz) + 3.0 * (y2 + z2) + 9.0 * uy * uz + 9.0 * (y2 * uz + uy * z2) + 9.0 * y2 * z2);
    f[18] = rho / 36.0 * (1.0 + 3.0 * (uy - uz) + 3.0 * (y2 + z2) - 9.0 * uy * uz + 9.0 * (-y2 * uz + uy * z2) + 9.0 * y2 * z2);
}

/* ------------------------------------------------------------------------ */
/* Eq. (eq:matrix): the central-moment basis, one row per monomial of the
 * shifted velocities cbar = c - u.  Row 18 is cbar_y^2 cbar_z^2 (the paper
 * prints cbar_y^2 cbar_y^2; the numeric matrix M of App. C has y^2 z^2 there).
 * T is row-major, T[row*19 + i]. */
void orc_T(double ux, double uy, double uz, double *T)
{
    for (int i = 0; i < Q; i++) {
        double a = CX[i] - ux, b = CY[i] - uy, c = CZ[i] - uz;
        double a2 = a * a, b2 = b * b, c2 = c * c;
        T[0 * Q + i] = 1.0;
        T[1 * Q + i] = a;
        T[2 * Q + i] = b;
        T[3 * Q + i] = c;
        T[4 * Q + i] = a2 + b2 + c2;
        T[5 * Q + i] = a2 - b2;
        T[6 * Q + i] = b2 - c2;
        T[7 * Q + i] = a * b;
        T[8 * Q + i] = a * c;
        T[9 * Q + i] = b * c;
        T[10 * Q + i] = a2 * b;
        T[11 * Q + i] = a * b2;
        T[12 * Q + i] = a2 * c;
        T[13 * Q + i] = a * c2;
        T[14 * Q + i] = b2 * c;
        T[15 * Q + i] = b * c2;
        T[16 * Q + i] = a2 * b2;
        T[17 * Q + i] = a2 * c2;
        T[18 * Q + i] = b2 * c2;
    }
}

static void matvec(const double *A, const double *x, double *y)
{
    for (int r = 0; r < Q; r++) {
        double s = 0.0;
        for (int c = 0; c < Q; c++) s += A[r * Q + c] * x[c];
        y[r] = s;
    }
}

/* Solve A x = b (n x n, row-major) by Gaussian elimination with partial
 * pivoting.  A and b are overwritten.  Returns 0, or -1 if A is singular. */
static int gauss_solve(int n, double *A, double *b, double *x)
{
    for (int k = 0; k < n; k++) {
        int p = k;
        double best = fabs(A[k * n + k]);
        for (int r = k + 1; r < n; r++) {
            double v = fabs(A[r * n + k]);
            if (v > best) {
                best = v;
                p = r;
            }
        }
        if (best == 0.0) return -1;
        if (p != k) {
            for (int c = 0; c < n; c++) {
                double t = A[k * n + c];
                A[k * n + c] = A[p * n + c];
                A[p * n + c] = t;
            }
            double t = b[k];
            b[k] = b[p];
            b[p] = t;
        }
        for (int r = k + 1; r < n; r++) {
            double m = A[r * n + k] / A[k * n + k];
            if (m == 0.0) continue;
            for (int c = k; c < n; c++) A[r * n + c] -= m * A[k * n + c];
            b[r] -= m * b[k];
        }
    }
    for (int k = n - 1; k >= 0; k--) {
        double s = b[k];
        for (int c = k + 1; c < n; c++) s -= A[k * n + c] * x[c];
        x[k] = s / A[k * n + k];
    }
    return 0;
}

int orc_solve19(const double *A, const double *b, double *x)
{
    double Ac[Q * Q], bc[Q];
    memcpy(Ac, A, sizeof(Ac));
    memcpy(bc, b, sizeof(bc));
    return gauss_solve(Q, Ac, bc, x);
}

/* ------------------------------------------------------------------------ */
/* App. B: velocity-space forcing term by moment matching.  The raw forcing
 * moments R^RM_pqr are those of Eq. (eq:RMQ19); they are placed on the rows of
 * M (the basis of Eq. (eq:matrix) at u = 0) and F_i = M^-1 R^RM is obtained
 * by a dense solve.  (The printed list Eq. (eq:FRMQ19) indexes directions in
 * an order other than Sec. II.A's, so it is not used.) */
void orc_forcing_rm(double ux, double uy, double uz, double Fx, double Fy, double Fz, double *R)
{
    double R000 = 0.0;
    double R100 = Fx, R010 = Fy, R001 = Fz;
    double R200 = 2.0 * ux * Fx, R020 = 2.0 * uy * Fy, R002 = 2.0 * uz * Fz;
    double R110 = ux * Fy + uy * Fx, R101 = ux * Fz + uz * Fx, R011 = uy * Fz + uz * Fy;
    double R210 = CS2 * Fy + ux * (ux * Fy + 2.0 * uy * Fx);
    double R120 = CS2 * Fx + uy * (uy * Fx + 2.0 * ux * Fy);
    double R201 = CS2 * Fz + ux * (ux * Fz + 2.0 * uz * Fx);
    double R102 = CS2 * Fx + uz * (uz * Fx + 2.0 * ux * Fz);
    double R021 = CS2 * Fz + uy * (uy * Fz + 2.0 * uz * Fy);
    double R012 = CS2 * Fy + uz * (uz * Fy + 2.0 * uy * Fz);
    double R220 = 2.0 * (ux * uy * (ux * Fy + uy * Fx) + CS2 * (ux * Fx + uy * Fy));
    double R202 = 2.0 * (ux * uz * (ux * Fz + uz * Fx) + CS2 * (ux * Fx + uz * Fz));
    double R022 = 2.0 * (uy * uz * (uy * Fz + uz * Fy) + CS2 * (uy * Fy + uz * Fz));
    /* rows of M: 1, cx, cy, cz, |c|^2, cx^2-cy^2, cy^2-cz^2, cxcy, cxcz, cycz,
     * cx^2cy, cxcy^2, cx^2cz, cxcz^2, cy^2cz, cycz^2, cx^2cy^2, cx^2cz^2, cy^2cz^2 */
    R[0] = R000;
    R[1] = R100;
    R[2] = R010;
    R[3] = R001;
    R[4] = R200 + R020 + R002;
    R[5] = R200 - R020;
    R[6] = R020 - R002;
    R[7] = R110;
    R[8] = R101;
    R[9] = R011;
    R[10] = R210;
    R[11] = R120;
    R[12] = R201;
    R[13] = R102;
    R[14] = R021;
    R[15] = R012;
    R[16] = R220;
    R[17] = R202;
    R[18] = R022;
}

void orc_forcing_pop(double ux, double uy, double uz, double Fx, double Fy, double Fz, double *Fi)
{
    double M[Q * Q], R[Q];
    orc_T(0.0, 0.0, 0.0, M);
    orc_forcing_rm(ux, uy, uz, Fx, Fy, Fz, R);
    orc_solve19(M, R, Fi);
}

/* App. E: the colour-gradient weights phi_i(alpha) (Eq. eq:varphi_ik). */
static double cgm_phi(int i, double alpha)
{
    int n2 = CX[i] * CX[i] + CY[i] * CY[i] + CZ[i] * CZ[i];
    if (n2 == 0) return alpha;
    if (n2 == 1) return (1.0 - alpha) / 12.0;
    return (1.0 - alpha) / 24.0;
}

/* App. E, Eq. (eq:feqCG): h_eq = f_eq + rho (phi_i - w_i). */
void orc_heq(double rho, double ux, double uy, double uz, double alpha, double *h)
{
    orc_feq(rho, ux, uy, uz, h);
    for (int i = 0; i < Q; i++) h[i] += rho * (cgm_phi(i, alpha) - weight(i));
}

/* ------------------------------------------------------------------------ */
/* Oracle-A.  Definition of the forced CM collision, Eq. (eq:posColl0):
 *   k* = (I - K) T f + K T h_eq + (I - K/2) T F_i,   T f* = k*.
 * K = diag[1,1,1,1, omega_b, omega x5, omega_3 x6, omega_4 x3] (Sec. II.B,
 * with the paper's choice omega_b = omega_3 = omega_4 = 1).  For the
 * colour-gradient model (cgm != 0) the equilibrium is h_eq of App. E. */
int orc_collide_dense(const double *f, double rho, double ux, double uy, double uz, double Fx, double Fy,
                      double Fz, double omega, double omega_b, double omega_3, double omega_4, int cgm,
                      double alpha, double *fout)
{
    double T[Q * Q], k[Q], keq[Q], R[Q], ks[Q], feq[Q], Fi[Q], Kd[Q];
    orc_T(ux, uy, uz, T);
    matvec(T, f, k);
    if (cgm)
        orc_heq(rho, ux, uy, uz, alpha, feq);
    else
        orc_feq(rho, ux, uy, uz, feq);
    matvec(T, feq, keq);
    orc_forcing_pop(ux, uy, uz, Fx, Fy, Fz, Fi);
    matvec(T, Fi, R);
    for (int r = 0; r < Q; r++) Kd[r] = 1.0;
    Kd[4] = omega_b;
    for (int r = 5; r <= 9; r++) Kd[r] = omega;
    for (int r = 10; r <= 15; r++) Kd[r] = omega_3;
    for (int r = 16; r <= 18; r++) Kd[r] = omega_4;
    for (int r = 0; r < Q; r++) ks[r] = (1.0 - Kd[r]) * k[r] + Kd[r] * keq[r] + (1.0 - 0.5 * Kd[r]) * R[r];
    return orc_solve19(T, ks, fout);
}

/* ------------------------------------------------------------------------ */
/* Oracle-B.  Post-collision central moments.
 * Single phase, Sec. II.B (forced list after Eq. eq:posColl0):
 *   k0* = rho, k1..3* = F/2, k4* = 3 rho cs^2, k5..9* = (1-omega) k5..9,
 *   k10* = Fy cs^2/2, k11* = Fx cs^2/2, k12* = Fz cs^2/2, k13* = Fx cs^2/2,
 *   k14* = Fz cs^2/2, k15* = Fy cs^2/2, k16..18* = rho cs^4.
 * Pre-collision k5..9 are the central second moments of f (Eq.
 * pre_collision_central_moments), computed here as plain sums over i. */
static void central_second_moments(const double *f, double ux, double uy, double uz, double *k59)
{
    double k5 = 0, k6 = 0, k7 = 0, k8 = 0, k9 = 0;
    for (int i = 0; i < Q; i++) {
        double a = CX[i] - ux, b = CY[i] - uy, c = CZ[i] - uz;
        k5 += f[i] * (a * a - b * b);
        k6 += f[i] * (b * b - c * c);
        k7 += f[i] * a * b;
        k8 += f[i] * a * c;
        k9 += f[i] * b * c;
    }
    k59[0] = k5;
    k59[1] = k6;
    k59[2] = k7;
    k59[3] = k8;
    k59[4] = k9;
}

void orc_kstar_fluid(const double *f, double rho, double ux, double uy, double uz, double Fx, double Fy, double Fz,
                     double omega, double *ks)
{
    double k59[5];
    central_second_moments(f, ux, uy, uz, k59);
    ks[0] = rho;
    ks[1] = Fx / 2.0;
    ks[2] = Fy / 2.0;
    ks[3] = Fz / 2.0;
    ks[4] = 3.0 * rho * CS2;
    for (int r = 0; r < 5; r++) ks[5 + r] = (1.0 - omega) * k59[r];
    ks[10] = Fy * CS2 / 2.0;
    ks[11] = Fx * CS2 / 2.0;
    ks[12] = Fz * CS2 / 2.0;
    ks[13] = Fx * CS2 / 2.0;
    ks[14] = Fz * CS2 / 2.0;
    ks[15] = Fy * CS2 / 2.0;
    ks[16] = rho * CS2 * CS2;
    ks[17] = rho * CS2 * CS2;
    ks[18] = rho * CS2 * CS2;
}

/* App. E post-collision CMs of the colour-gradient single-phase operator.
 * k16..18 carry a factor 1/6 that the printed list omits: T h_eq gives
 * rho [1 + ux^2 + uy^2 - alpha (1 + 3ux^2 + 3uy^2)] / 6, which equals
 * rho cs^4 at alpha = 1/3, u = 0 as the single-phase list requires. */
void orc_kstar_cgm(const double *f, double rho, double ux, double uy, double uz, double Fx, double Fy, double Fz,
                   double omega, double alpha, double *ks)
{
    double k59[5];
    central_second_moments(f, ux, uy, uz, k59);
    double a3 = (3.0 * alpha - 1.0) / 6.0;
    ks[0] = rho;
    ks[1] = Fx / 2.0;
    ks[2] = Fy / 2.0;
    ks[3] = Fz / 2.0;
    ks[4] = 3.0 * rho * (1.0 - alpha) / 2.0;
    for (int r = 0; r < 5; r++) ks[5 + r] = (1.0 - omega) * k59[r];
    ks[10] = Fy * CS2 / 2.0 + rho * uy * a3;
    ks[11] = Fx * CS2 / 2.0 + rho * ux * a3;
    ks[12] = Fz * CS2 / 2.0 + rho * uz * a3;
    ks[13] = Fx * CS2 / 2.0 + rho * ux * a3;
    ks[14] = Fz * CS2 / 2.0 + rho * uz * a3;
    ks[15] = Fy * CS2 / 2.0 + rho * uy * a3;
    ks[16] = rho * (1.0 + ux * ux + uy * uy - alpha * (1.0 + 3.0 * ux * ux + 3.0 * uy * uy)) / 6.0;
    ks[17] = rho * (1.0 + ux * ux + uz * uz - alpha * (1.0 + 3.0 * ux * ux + 3.0 * uz * uz)) / 6.0;
    ks[18] = rho * (1.0 + uy * uy + uz * uz - alpha * (1.0 + 3.0 * uy * uy + 3.0 * uz * uz)) / 6.0;
}

/* App. C, Eq. (pdfQ19): populations from raw moments, f = M^-1 r. */
static void raw_to_populations(const double *r, double *f)
{
    f[0] = r[0] - r[4] + r[16] + r[17] + r[18];
    f[1] = (r[11] + r[13] - r[1] - r[16] - r[17]) / 2.0 + (r[4] + 2.0 * r[5] + r[6]) * CS2 / 2.0;
    f[2] = (r[10] + r[15] - r[2] - r[16] - r[18]) / 2.0 + (r[4] + r[6] - r[5]) * CS2 / 2.0;
    f[3] = (r[12] + r[14] - r[3] - r[17] - r[18]) / 2.0 + (r[4] - r[5] - 2.0 * r[6]) * CS2 / 2.0;
    f[4] = (r[7] + r[16] - r[10] - r[11]) / 4.0;
    f[5] = (r[10] + r[16] - r[7] - r[11]) / 4.0;
    f[6] = (r[8] + r[17] - r[12] - r[13]) / 4.0;
    f[7] = (r[12] + r[17] - r[8] - r[13]) / 4.0;
    f[8] = (r[9] + r[18] - r[14] - r[15]) / 4.0;
    f[9] = (r[14] + r[18] - r[9] - r[15]) / 4.0;
    f[10] = (r[1] - r[11] - r[13] - r[16] - r[17]) / 2.0 + (r[4] + 2.0 * r[5] + r[6]) * CS2 / 2.0;
    f[11] = (r[2] - r[10] - r[15] - r[16] - r[18]) / 2.0 + (r[4] + r[6] - r[5]) * CS2 / 2.0;
    f[12] = (r[3] - r[12] - r[14] - r[17] - r[18]) / 2.0 + (r[4] - r[5] - 2.0 * r[6]) * CS2 / 2.0;
    f[13] = (r[7] + r[10] + r[11] + r[16]) / 4.0;
    f[14] = (r[11] + r[16] - r[7] - r[10]) / 4.0;
    f[15] = (r[8] + r[12] + r[13] + r[17]) / 4.0;
    f[16] = (r[13] + r[17] - r[8] - r[12]) / 4.0;
    f[17] = (r[9] + r[14] + r[15] + r[18]) / 4.0;
    f[18] = (r[15] + r[18] - r[9] - r[14]) / 4.0;
}

/* App. C two-step reconstruction.  r* = N^-1 k* (Eq. rawQ19), then
 * f* = M^-1 r* (Eq. pdfQ19).  Corrections to the printed text:
 *   r16*: the k5* term carries c_s^2, (2uy^2 - ux^2) k5* cs^2;
 *   r17*: the k5* term carries c_s^2, (2uz^2 - ux^2) k5* cs^2;
 *   r18*: the k6* term carries c_s^2, (uz^2 - 2uy^2) k6* cs^2;
 *   f3*:  the printed "(r4 - r5 - 2 - r6)" is (r4 - r5 - 2 r6), the same
 *         combination as in f12*, which the paper prints as (r4 - r5 - r6);
 *         both read (r4 - r5 - 2 r6) cs^2 / 2.
 * (Each correction follows from expanding c = cbar + u in the raw monomial
 * and writing sum f cbar_x^2 etc. through k4, k5, k6; the dense Oracle-A
 * checks all of them.) */
void orc_back_transform(double rho, double ux, double uy, double uz, const double *k, double *f)
{
    double x2 = ux * ux, y2 = uy * uy, z2 = uz * uz;
    double r[Q];
    r[0] = rho;
    r[1] = rho * ux + k[1];
    r[2] = rho * uy + k[2];
    r[3] = rho * uz + k[3];
    r[4] = rho * (x2 + y2 + z2) + 2.0 * ux * k[1] + 2.0 * uy * k[2] + 2.0 * uz * k[3] + k[4];
    r[5] = rho * (x2 - y2) + 2.0 * ux * k[1] - 2.0 * uy * k[2] + k[5];
    r[6] = rho * (y2 - z2) + 2.0 * uy * k[2] - 2.0 * uz * k[3] + k[6];
    r[7] = rho * ux * uy + uy * k[1] + ux * k[2] + k[7];
    r[8] = rho * ux * uz + uz * k[1] + ux * k[3] + k[8];
    r[9] = rho * uy * uz + uz * k[2] + uy * k[3] + k[9];
    r[10] = rho * x2 * uy + 2.0 * ux * uy * k[1] + x2 * k[2] + uy * k[4] * CS2 + 2.0 * uy * k[5] * CS2 +
            uy * k[6] * CS2 + 2.0 * ux * k[7] + k[10];
    r[11] = rho * ux * y2 + y2 * k[1] + 2.0 * ux * uy * k[2] + ux * k[4] * CS2 - ux * k[5] * CS2 + ux * k[6] * CS2 +
            2.0 * uy * k[7] + k[11];
    r[12] = rho * x2 * uz + 2.0 * ux * uz * k[1] + x2 * k[3] + uz * k[4] * CS2 + 2.0 * uz * k[5] * CS2 +
            uz * k[6] * CS2 + 2.0 * ux * k[8] + k[12];
    r[13] = rho * ux * z2 + z2 * k[1] + 2.0 * ux * uz * k[3] + ux * k[4] * CS2 - ux * k[5] * CS2 -
            2.0 * ux * k[6] * CS2 + 2.0 * uz * k[8] + k[13];
    r[14] = rho * y2 * uz + 2.0 * uy * uz * k[2] + y2 * k[3] + uz * k[4] * CS2 - uz * k[5] * CS2 + uz * k[6] * CS2 +
            2.0 * uy * k[9] + k[14];
    r[15] = rho * uy * z2 + z2 * k[2] + 2.0 * uy * uz * k[3] + uy * k[4] * CS2 - uy * k[5] * CS2 -
            2.0 * uy * k[6] * CS2 + 2.0 * uz * k[9] + k[15];
    r[16] = rho * x2 * y2 + 2.0 * ux * y2 * k[1] + 2.0 * x2 * uy * k[2] + (x2 + y2) * k[4] * CS2 +
            (2.0 * y2 - x2) * k[5] * CS2 + (x2 + y2) * k[6] * CS2 + 4.0 * ux * uy * k[7] + 2.0 * uy * k[10] +
            2.0 * ux * k[11] + k[16];
    r[17] = rho * x2 * z2 + 2.0 * ux * z2 * k[1] + 2.0 * x2 * uz * k[3] + (x2 + z2) * k[4] * CS2 +
            (2.0 * z2 - x2) * k[5] * CS2 + (z2 - 2.0 * x2) * k[6] * CS2 + 4.0 * ux * uz * k[8] + 2.0 * uz * k[12] +
            2.0 * ux * k[13] + k[17];
    r[18] = rho * y2 * z2 + 2.0 * uy * z2 * k[2] + 2.0 * y2 * uz * k[3] + (y2 + z2) * k[4] * CS2 +
            (-y2 - z2) * k[5] * CS2 + (z2 - 2.0 * y2) * k[6] * CS2 + 4.0 * uy * uz * k[9] + 2.0 * uz * k[14] +
            2.0 * uy * k[15] + k[18];

    raw_to_populations(r, f);
}

/* App. C, raw-moment variant (N = I, T = M): the printed post-collision list
 *   k0* = rho, k1..3* = rho u + F/2, k4* = rho (3 cs^2 + |u|^2),
 *   k5..9* = (1 - omega) k5..9 + omega k5..9_eq (raw second moments of f),
 *   k10* = Fy cs^2/2 + rho uy (ux^2 + cs^2), ... (third order at equilibrium
 *   plus cs^2 F/2), k16..18* = rho (ua^2 + cs^2)(ub^2 + cs^2),
 * with r* = k*, then f* = M^-1 r*.  Unlike the central form, the printed list
 * carries no velocity-dependent forcing terms at second and higher order; with
 * F = 0 it is the raw-moment MRT with the same relaxation matrix. */
void orc_kstar_rm(const double *f, double rho, double ux, double uy, double uz, double Fx, double Fy, double Fz,
                  double omega, double *ks)
{
    double k5 = 0, k6 = 0, k7 = 0, k8 = 0, k9 = 0;
    for (int i = 0; i < Q; i++) {
        k5 += f[i] * (CX[i] * CX[i] - CY[i] * CY[i]);
        k6 += f[i] * (CY[i] * CY[i] - CZ[i] * CZ[i]);
        k7 += f[i] * CX[i] * CY[i];
        k8 += f[i] * CX[i] * CZ[i];
        k9 += f[i] * CY[i] * CZ[i];
    }
    double x2 = ux * ux, y2 = uy * uy, z2 = uz * uz;
    ks[0] = rho;
    ks[1] = Fx / 2.0 + rho * ux;
    ks[2] = Fy / 2.0 + rho * uy;
    ks[3] = Fz / 2.0 + rho * uz;
    ks[4] = rho * (3.0 * CS2 + x2 + y2 + z2);
    ks[5] = (1.0 - omega) * k5 + omega * rho * (x2 - y2);
    ks[6] = (1.0 - omega) * k6 + omega * rho * (y2 - z2);
    ks[7] = (1.0 - omega) * k7 + omega * rho * ux * uy;
    ks[8] = (1.0 - omega) * k8 + omega * rho * ux * uz;
    ks[9] = (1.0 - omega) * k9 + omega * rho * uy * uz;
    ks[10] = Fy * CS2 / 2.0 + rho * uy * (x2 + CS2);
    ks[11] = Fx * CS2 / 2.0 + rho * ux * (y2 + CS2);
    ks[12] = Fz * CS2 / 2.0 + rho * uz * (x2 + CS2);
    ks[13] = Fx * CS2 / 2.0 + rho * ux * (z2 + CS2);
    ks[14] = Fz * CS2 / 2.0 + rho * uz * (y2 + CS2);
    ks[15] = Fy * CS2 / 2.0 + rho * uy * (z2 + CS2);
    ks[16] = rho * (x2 + CS2) * (y2 + CS2);
    ks[17] = rho * (x2 + CS2) * (z2 + CS2);
    ks[18] = rho * (y2 + CS2) * (z2 + CS2);
}

void orc_collide_rm(const double *f, double rho, double ux, double uy, double uz, double Fx, double Fy, double Fz,
                    double omega, double *fout)
{
    double ks[Q];
    orc_kstar_rm(f, rho, ux, uy, uz, Fx, Fy, Fz, omega, ks);
    raw_to_populations(ks, fout);
}

/* The raw-moment MRT by definition: k = M f, k_eq = M f_eq, R = M F_i with the
 * printed raw forcing moments (App. B), k* = (I - K) k + K k_eq + (I - K/2) R,
 * then M f* = k* solved; M = T(0) (App. C). */
int orc_collide_dense_rm(const double *f, double rho, double ux, double uy, double uz, double Fx, double Fy, double Fz,
                         double omega, double *fout)
{
    double M[Q * Q], k[Q], keq[Q], R[Q], ks[Q], feq[Q], Kd[Q];
    orc_T(0.0, 0.0, 0.0, M);
    matvec(M, f, k);
    orc_feq(rho, ux, uy, uz, feq);
    matvec(M, feq, keq);
    orc_forcing_rm(ux, uy, uz, Fx, Fy, Fz, R);
    for (int r = 0; r < Q; r++) Kd[r] = (r >= 5 && r <= 9) ? omega : 1.0;
    for (int r = 0; r < Q; r++) ks[r] = (1.0 - Kd[r]) * k[r] + Kd[r] * keq[r] + (1.0 - 0.5 * Kd[r]) * R[r];
    return orc_solve19(M, ks, fout);
}

int orc_collide_closed(const double *f, double rho, double ux, double uy, double uz, double Fx, double Fy,
                       double Fz, double omega, int cgm, double alpha, double *fout)
{
    double ks[Q];
    if (cgm)
        orc_kstar_cgm(f, rho, ux, uy, uz, Fx, Fy, Fz, omega, alpha, ks);
    else
        orc_kstar_fluid(f, rho, ux, uy, uz, Fx, Fy, Fz, omega, ks);
    orc_back_transform(rho, ux, uy, uz, ks, fout);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Magnetic field (Sec. III.F cites Dellar 2002 without restating it; this is
 * the reading used): vector-valued BGK populations g_{m,a} on D3Q7,
 * b = sum_m g_m, equilibrium g_eq_{m,a} = w_m [b_a + c_{m,b}(u_b b_a - b_b u_a)
 * / cs_m^2], w = 1/4 (rest), 1/8 (axes), cs_m^2 = 1/4, eta = cs_m^2 (tau_m - 1/2).
 * The current j = curl b follows from the antisymmetric part of the
 * non-equilibrium flux Lambda_{ba} = sum_m c_{m,b} g_{m,a}:
 *   j_c = -eps_{cba} (Lambda - Lambda_eq)_{ba} / (tau_m cs_m^2).
 * Storage g[cell*21 + m*3 + a]. */
static const int MX[QM] = {0, 1, -1, 0, 0, 0, 0};
static const int MY[QM] = {0, 0, 0, 1, -1, 0, 0};
static const int MZ[QM] = {0, 0, 0, 0, 0, 1, -1};
static const double CSM2 = 0.25;

static double mweight(int m) { return m == 0 ? 0.25 : 0.125; }
static int mopposite(int m) { return m == 0 ? 0 : (m % 2 == 1 ? m + 1 : m - 1); }

void orc_geq(double ux, double uy, double uz, double bx, double by, double bz, double *g)
{
    double u[3] = {ux, uy, uz}, b[3] = {bx, by, bz};
    for (int m = 0; m < QM; m++) {
        int c[3] = {MX[m], MY[m], MZ[m]};
        for (int a = 0; a < 3; a++) {
            double s = b[a];
            for (int bb = 0; bb < 3; bb++) s += c[bb] * (u[bb] * b[a] - b[bb] * u[a]) / CSM2;
            g[m * 3 + a] = mweight(m) * s;
        }
    }
}

/* Lorentz force from the gathered magnetic populations and the uncorrected
 * velocity ustar = sum f c / rho (explicit reading: the equilibrium flux in
 * j uses ustar; the F/2 correction of u follows from F). */
void orc_current(const double *g, double ux, double uy, double uz, double tau_m, double *bout, double *j)
{
    double b[3] = {0, 0, 0}, L[3][3] = {{0}};
    double u[3] = {ux, uy, uz};
    for (int m = 0; m < QM; m++) {
        int c[3] = {MX[m], MY[m], MZ[m]};
        for (int a = 0; a < 3; a++) {
            b[a] += g[m * 3 + a];
            for (int bb = 0; bb < 3; bb++) L[bb][a] += c[bb] * g[m * 3 + a];
        }
    }
    double N[3][3];
    for (int bb = 0; bb < 3; bb++)
        for (int a = 0; a < 3; a++) N[bb][a] = L[bb][a] - (u[bb] * b[a] - b[bb] * u[a]);
    double s = -1.0 / (tau_m * CSM2);
    /* j_x = eps_xyz N_yz + eps_xzy N_zy = N_yz - N_zy, cyclic. */
    j[0] = s * (N[1][2] - N[2][1]);
    j[1] = s * (N[2][0] - N[0][2]);
    j[2] = s * (N[0][1] - N[1][0]);
    for (int a = 0; a < 3; a++) bout[a] = b[a];
}

/* ------------------------------------------------------------------------ */
/* Domain-level driver. */
typedef struct {
    int nx, ny, nz;
    int periodic[3]; /* 1 = periodic axis, 0 = walls at both ends */
    double lid_u[3]; /* velocity of the +y wall (Ladd's moving-wall term, rho_w = 1) */
    double omega, omega_b, omega_3, omega_4;
    double g[3];     /* body acceleration, F = rho g */
    int physics;     /* 0 single phase, 1 MHD, 2 colour gradient, 3 Shan-Chen */
    int closed_form; /* 0: Oracle-A (dense), 1: Oracle-B (two-step closed form) */
    double tau_m;    /* MHD: magnetic relaxation time */
    double b_wall[3];
    double alpha_r, alpha_b, A, beta; /* CGM */
    int nthreads;
    double G; /* Shan-Chen interaction strength (physics 3) */
    double rho_ref; /* body force F = (rho - rho_ref) g (Sec. III.H uses the mean density) */
    int wall_model; /* 0: half-way bounce-back; 1: regularized on-node walls on the y axis */
    int raw_moments; /* 1: the raw-moment variant of App. C (N = I) instead of central moments */
} orc_params;

static long cell_index(const orc_params *p, int x, int y, int z)
{
    return (long)x + (long)p->nx * ((long)y + (long)p->ny * (long)z);
}

/* Neighbour coordinate along one axis: returns -1 if it leaves the domain
 * through a wall. */
static int wrap(int v, int n, int periodic)
{
    if (v >= 0 && v < n) return v;
    if (!periodic) return -1;
    return ((v % n) + n) % n;
}

/* Regularized on-node wall (Sec. III opening paragraph cites Latt, Chopard,
 * Malaspinas, Deville and Michler, Phys. Rev. E 77, 056703 (2008), "straight
 * velocity boundaries"): the wall lies on the boundary node, whose velocity is
 * the wall's.  fin holds the pulled populations; those with c_y = sgn (sgn the
 * y component of the inward normal: +1 at y = 0, -1 at y = ny - 1) came from
 * outside and are unknown.
 *  1. rho from the known ones: the normal momentum of the bare populations is
 *     rho u_n - F_n/2 (rho u = Sum f c + F/2, F = (rho - rho_ref) g), so
 *     rho (1 - u_n + g_n/2) = rho_0 + 2 rho_out + rho_ref g_n/2, rho_0 the sum
 *     over c_y = 0 and rho_out over c_y = -sgn;
 *  2. f_eq = the extended equilibrium at rho and u_eq = u_w - F/(2 rho), so that
 *     the corrected velocity equals u_w;
 *  3. unknown populations: bounce-back of the non-equilibrium part,
 *     f_i = f_eq_i + f_opp(i) - f_eq_opp(i);
 *  4. Pi_neq = Sum_i c_i c_i (f_i - f_eq_i) over all 19;
 *  5. every population is replaced by f_eq_i + w_i/(2 cs^4) Q_i : Pi_neq,
 *     Q_i = c_i c_i - cs^2 I. */
void orc_regularize(double *fin, int sgn, const double *u_w, const double *g, double rho_ref)
{
    double rho0 = 0, rout = 0;
    for (int i = 0; i < Q; i++) {
        if (CY[i] == 0) rho0 += fin[i];
        if (CY[i] == -sgn) rout += fin[i];
    }
    double gn = sgn * g[1], un = sgn * u_w[1];
    double rho = (rho0 + 2.0 * rout + 0.5 * rho_ref * gn) / (1.0 - un + 0.5 * gn);
    double ueq[3], feq[Q], pi[3][3] = {{0}};
    for (int a = 0; a < 3; a++) ueq[a] = u_w[a] - 0.5 * (rho - rho_ref) * g[a] / rho;
    orc_feq(rho, ueq[0], ueq[1], ueq[2], feq);
    for (int i = 0; i < Q; i++)
        if (CY[i] == sgn) fin[i] = feq[i] + fin[opposite(i)] - feq[opposite(i)];
    for (int i = 0; i < Q; i++) {
        double c[3] = {CX[i], CY[i], CZ[i]}, d = fin[i] - feq[i];
        for (int a = 0; a < 3; a++)
            for (int b = 0; b < 3; b++) pi[a][b] += c[a] * c[b] * d;
    }
    double tr = pi[0][0] + pi[1][1] + pi[2][2];
    for (int i = 0; i < Q; i++) {
        double c[3] = {CX[i], CY[i], CZ[i]}, qp = -CS2 * tr;
        for (int a = 0; a < 3; a++)
            for (int b = 0; b < 3; b++) qp += c[a] * c[b] * pi[a][b];
        fin[i] = feq[i] + weight(i) / (2.0 * CS2 * CS2) * qp;
    }
}

/* Streaming, Eq. (streaming), in gather form: f_i(x, t+1) = f*_i(x - c_i, t).
 * A source outside the domain through a wall gives half-way bounce-back,
 * f_i(x) = f*_opp(i)(x) + 2 w_i rho_w (c_i . u_w)/cs^2 with rho_w = 1, u_w the
 * lid velocity when the source lies beyond the +y face, else 0. */
static void gather_f(const orc_params *p, const double *fpost, int x, int y, int z, double *fin, int lid_term)
{
    long self = cell_index(p, x, y, z);
    for (int i = 0; i < Q; i++) {
        int sx = wrap(x - CX[i], p->nx, p->periodic[0]);
        int sy = wrap(y - CY[i], p->ny, p->periodic[1]);
        int sz = wrap(z - CZ[i], p->nz, p->periodic[2]);
        if (sx >= 0 && sy >= 0 && sz >= 0) {
            fin[i] = fpost[cell_index(p, sx, sy, sz) * Q + i];
        } else {
            double v = fpost[self * Q + opposite(i)];
            if (lid_term && !p->periodic[1] && y - CY[i] >= p->ny) {
                double cu = CX[i] * p->lid_u[0] + CY[i] * p->lid_u[1] + CZ[i] * p->lid_u[2];
                v += 2.0 * weight(i) * cu / CS2;
            }
            fin[i] = v;
        }
    }
    /* regularized walls replace the bounce-back values on the y boundary nodes */
    if (lid_term && p->wall_model == 1 && !p->periodic[1] && (y == 0 || y == p->ny - 1)) {
        const double rest[3] = {0.0, 0.0, 0.0};
        orc_regularize(fin, y == 0 ? 1 : -1, y == 0 ? rest : p->lid_u, p->g, p->rho_ref);
    }
}

/* Magnetic streaming with anti-bounce-back at walls: a population arriving
 * from beyond a wall is -g*_opp(x) + 2 w_m b_wall (Dirichlet b = b_wall at
 * the half-way wall, wall at rest). */
static void gather_g(const orc_params *p, const double *gpost, int x, int y, int z, double *gin)
{
    long self = cell_index(p, x, y, z);
    for (int m = 0; m < QM; m++) {
        int sx = wrap(x - MX[m], p->nx, p->periodic[0]);
        int sy = wrap(y - MY[m], p->ny, p->periodic[1]);
        int sz = wrap(z - MZ[m], p->nz, p->periodic[2]);
        for (int a = 0; a < 3; a++) {
            if (sx >= 0 && sy >= 0 && sz >= 0)
                gin[m * 3 + a] = gpost[cell_index(p, sx, sy, sz) * 21 + m * 3 + a];
            else
                gin[m * 3 + a] = -gpost[self * 21 + mopposite(m) * 3 + a] + 2.0 * mweight(m) * p->b_wall[a];
        }
    }
}

static void raw_moments(const double *f, double *rho, double *jx, double *jy, double *jz)
{
    double r = 0, a = 0, b = 0, c = 0;
    for (int i = 0; i < Q; i++) {
        r += f[i];
        a += f[i] * CX[i];
        b += f[i] * CY[i];
        c += f[i] * CZ[i];
    }
    *rho = r;
    *jx = a;
    *jy = b;
    *jz = c;
}

void orc_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int orc_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Sec. III.G: Shan-Chen pseudopotential psi = 1 - exp(-rho) and interaction
 * force F(x) = -G psi(x) sum_i w_i c_i psi(x + c_i) (no c_s^2 factor, as
 * printed).  psi holds the pseudopotential of every node computed from the
 * post-stream densities; a neighbour behind a wall contributes the node's own
 * psi. */
static void sc_force(const orc_params *p, const double *psi, int x, int y, int z, double *F)
{
    double own = psi[cell_index(p, x, y, z)];
    double sx = 0, sy = 0, sz = 0;
    for (int i = 1; i < Q; i++) {
        int nx_ = wrap(x + CX[i], p->nx, p->periodic[0]);
        int ny_ = wrap(y + CY[i], p->ny, p->periodic[1]);
        int nz_ = wrap(z + CZ[i], p->nz, p->periodic[2]);
        double v = (nx_ >= 0 && ny_ >= 0 && nz_ >= 0) ? psi[cell_index(p, nx_, ny_, nz_)] : own;
        sx += weight(i) * CX[i] * v;
        sy += weight(i) * CY[i] * v;
        sz += weight(i) * CZ[i] * v;
    }
    F[0] = -p->G * own * sx;
    F[1] = -p->G * own * sy;
    F[2] = -p->G * own * sz;
}

/* The Shan-Chen force of every node for a given pseudopotential field psi
 * (layout [nz][ny][nx]); F is [3][nz][ny][nx]. */
void orc_sc_force_field(const orc_params *p, const double *psi, double *F)
{
    long n = (long)p->nx * p->ny * p->nz;
    for (int z = 0; z < p->nz; z++)
        for (int y = 0; y < p->ny; y++)
            for (int x = 0; x < p->nx; x++) {
                long c = cell_index(p, x, y, z);
                double Fc[3];
                sc_force(p, psi, x, y, z, Fc);
                F[c] = Fc[0];
                F[n + c] = Fc[1];
                F[2 * n + c] = Fc[2];
            }
}

/* Per-node macroscopic state of a gathered set, shared by step and fields. */
typedef struct {
    double rho, u[3], F[3], b[3], j[3];
} node_state;

static void node_macro_sc(const orc_params *p, const double *fin, const double *gin, const double *psi, int x, int y,
                          int z, node_state *s);
static void node_macro(const orc_params *p, const double *fin, const double *gin, node_state *s)
{
    double jx, jy, jz;
    raw_moments(fin, &s->rho, &jx, &jy, &jz);
    double rho = s->rho;
    s->b[0] = s->b[1] = s->b[2] = 0.0;
    s->j[0] = s->j[1] = s->j[2] = 0.0;
    /* Body force F = (rho - rho_ref) g: a constant acceleration for rho_ref = 0;
     * the Rayleigh-Taylor test (Sec. III.H) takes rho_ref = (rho_h + rho_l)/2. */
    s->F[0] = (rho - p->rho_ref) * p->g[0];
    s->F[1] = (rho - p->rho_ref) * p->g[1];
    s->F[2] = (rho - p->rho_ref) * p->g[2];
    if (p->physics == 1 && gin) {
        double us[3] = {jx / rho, jy / rho, jz / rho};
        orc_current(gin, us[0], us[1], us[2], p->tau_m, s->b, s->j);
        /* Lorentz force F = j x b (Sec. III.F). */
        s->F[0] += s->j[1] * s->b[2] - s->j[2] * s->b[1];
        s->F[1] += s->j[2] * s->b[0] - s->j[0] * s->b[2];
        s->F[2] += s->j[0] * s->b[1] - s->j[1] * s->b[0];
    }
    /* rho u = sum f c + F/2 (App. E macroscopic variables). */
    s->u[0] = (jx + 0.5 * s->F[0]) / rho;
    s->u[1] = (jy + 0.5 * s->F[1]) / rho;
    s->u[2] = (jz + 0.5 * s->F[2]) / rho;
}

static int collide(const orc_params *p, const double *fin, const node_state *s, int cgm, double alpha,
                   double *fout)
{
    if (p->raw_moments && !cgm) {
        if (p->closed_form) {
            orc_collide_rm(fin, s->rho, s->u[0], s->u[1], s->u[2], s->F[0], s->F[1], s->F[2], p->omega, fout);
            return 0;
        }
        return orc_collide_dense_rm(fin, s->rho, s->u[0], s->u[1], s->u[2], s->F[0], s->F[1], s->F[2], p->omega,
                                    fout);
    }
    if (p->closed_form)
        return orc_collide_closed(fin, s->rho, s->u[0], s->u[1], s->u[2], s->F[0], s->F[1], s->F[2], p->omega, cgm,
                                  alpha, fout);
    return orc_collide_dense(fin, s->rho, s->u[0], s->u[1], s->u[2], s->F[0], s->F[1], s->F[2], p->omega,
                             p->omega_b, p->omega_3, p->omega_4, cgm, alpha, fout);
}

/* Macroscopic state with the Shan-Chen force added to the body force. */
static void node_macro_sc(const orc_params *p, const double *fin, const double *gin, const double *psi, int x, int y,
                          int z, node_state *s)
{
    double jx, jy, jz, Fsc[3];
    (void)gin;
    raw_moments(fin, &s->rho, &jx, &jy, &jz);
    sc_force(p, psi, x, y, z, Fsc);
    for (int a = 0; a < 3; a++) {
        s->F[a] = (s->rho - p->rho_ref) * p->g[a] + Fsc[a];
        s->b[a] = s->j[a] = 0.0;
    }
    s->u[0] = (jx + 0.5 * s->F[0]) / s->rho;
    s->u[1] = (jy + 0.5 * s->F[1]) / s->rho;
    s->u[2] = (jz + 0.5 * s->F[2]) / s->rho;
}

/* Pseudopotential of every node from the gathered (post-stream) densities. */
static void sc_pseudopotential(const orc_params *p, const double *f, double *psi)
{
    int nx = p->nx, ny = p->ny, nz = p->nz;
#pragma omp parallel for schedule(static)
    for (int z = 0; z < nz; z++)
        for (int y = 0; y < ny; y++)
            for (int x = 0; x < nx; x++) {
                double fin[Q], rho = 0;
                gather_f(p, f, x, y, z, fin, 1);
                for (int i = 0; i < Q; i++) rho += fin[i];
                psi[cell_index(p, x, y, z)] = 1.0 - exp(-rho);
            }
}

/* Initial state: populations at the equilibrium of the given fields (Sec.
 * III opening paragraph).  Single phase and MHD: f = f_eq(rho,u); MHD also
 * g = g_eq(u, b).  CGM: the total f = h_eq(rho, u, alpha) with
 * rho_r = rho (1+phase)/2, rho_b = rho (1-phase)/2, split by colour fraction. */
int orc_init(const orc_params *p, const double *rho, const double *u, const double *phase, const double *B,
             double *f, double *g, double *fr, double *fb)
{
    long n = (long)p->nx * p->ny * p->nz;
    for (long c = 0; c < n; c++) {
        double ux = u[c], uy = u[n + c], uz = u[2 * n + c];
        if (p->physics == 2) {
            double rr = rho[c] * (1.0 + phase[c]) / 2.0, rb = rho[c] * (1.0 - phase[c]) / 2.0;
            double alpha = (rr * p->alpha_r + rb * p->alpha_b) / rho[c];
            double h[Q];
            orc_heq(rho[c], ux, uy, uz, alpha, h);
            for (int i = 0; i < Q; i++) {
                fr[c * Q + i] = rr / rho[c] * h[i];
                fb[c * Q + i] = rb / rho[c] * h[i];
            }
        } else {
            orc_feq(rho[c], ux, uy, uz, f + c * Q);
            if (p->physics == 1) orc_geq(ux, uy, uz, B[c], B[n + c], B[2 * n + c], g + c * 21);
        }
    }
    return 0;
}

static void cgm_gradient(const orc_params *p, const double *phi, int x, int y, int z, double *grad)
{
    double gx = 0, gy = 0, gz = 0;
    double own = phi[cell_index(p, x, y, z)];
    for (int i = 1; i < Q; i++) {
        int sx = wrap(x + CX[i], p->nx, p->periodic[0]);
        int sy = wrap(y + CY[i], p->ny, p->periodic[1]);
        int sz = wrap(z + CZ[i], p->nz, p->periodic[2]);
        double v = (sx >= 0 && sy >= 0 && sz >= 0) ? phi[cell_index(p, sx, sy, sz)] : own;
        gx += weight(i) * CX[i] * v;
        gy += weight(i) * CY[i] * v;
        gz += weight(i) * CZ[i] * v;
    }
    grad[0] = gx / CS2;
    grad[1] = gy / CS2;
    grad[2] = gz / CS2;
}

/* App. E perturbation operator (Eq. eq:perturb) with the squared projection
 * (c_i . grad phi)^2, the form that conserves mass.  Each colour k receives
 * (A_k/2)|grad phi|[...]; with A_r = A_b = A both act on the total
 * post-collision populations as A |grad phi| [...], the amplitude for which
 * sigma = (2/9)(A_r + A_b)/omega = (4/9) A/omega (App. E). */
void orc_cgm_perturb(const double *grad, double A, double *f)
{
    double n2 = grad[0] * grad[0] + grad[1] * grad[1] + grad[2] * grad[2];
    if (n2 <= 1e-24) return;
    double nrm = sqrt(n2);
    for (int i = 0; i < Q; i++) {
        double cg = CX[i] * grad[0] + CY[i] * grad[1] + CZ[i] * grad[2];
        int c2 = CX[i] * CX[i] + CY[i] * CY[i] + CZ[i] * CZ[i];
        double Bi = c2 == 0 ? -1.0 / 3.0 : (c2 == 1 ? 1.0 / 18.0 : 1.0 / 36.0);
        f[i] += A * nrm * (weight(i) * cg * cg / n2 - Bi);
    }
}

/* App. E recolouring (Eqs. eq:op3r, eq:op3b) with g_eq(rho, 0) = rho phi_i(alpha)
 * and cos(theta_i) = c_i . grad phi / (|c_i| |grad phi|) (0 for the rest
 * direction or a vanishing gradient). */
void orc_cgm_recolour(const double *f, const double *grad, double rho_r, double rho_b, double alpha, double beta,
                      double *fr, double *fb)
{
    double rho = rho_r + rho_b;
    double n = sqrt(grad[0] * grad[0] + grad[1] * grad[1] + grad[2] * grad[2]);
    for (int i = 0; i < Q; i++) {
        double cos_t = 0.0;
        int c2 = CX[i] * CX[i] + CY[i] * CY[i] + CZ[i] * CZ[i];
        if (c2 > 0 && n > 1e-12) cos_t = (CX[i] * grad[0] + CY[i] * grad[1] + CZ[i] * grad[2]) / (sqrt((double)c2) * n);
        double geq = rho * cgm_phi(i, alpha);
        double sep = beta * rho_r * rho_b / (rho * rho) * cos_t * geq;
        fr[i] = rho_r / rho * f[i] + sep;
        fb[i] = rho_b / rho * f[i] - sep;
    }
}

/* One or more time steps.  f/ftmp (single phase, MHD), g/gtmp (MHD),
 * fr/fb/frtmp/fbtmp/phi (CGM); the result is left in f (g, fr, fb). */
int orc_step(const orc_params *p, double *f, double *ftmp, double *g, double *gtmp, double *fr, double *fb,
             double *frtmp, double *fbtmp, double *phi, long nsteps)
{
    int nx = p->nx, ny = p->ny, nz = p->nz;
    long n = (long)nx * ny * nz;
    int err = 0;
    for (long s = 0; s < nsteps; s++) {
        if (p->physics == 2) {
            /* Pass 1: post-stream colour densities and the order parameter
             * phi = (rho_r - rho_b)/(rho_r + rho_b) (Eq. eq:order). */
#pragma omp parallel for schedule(static)
            for (int z = 0; z < nz; z++)
                for (int y = 0; y < ny; y++)
                    for (int x = 0; x < nx; x++) {
                        double a[Q], b[Q], rr = 0, rb = 0;
                        gather_f(p, fr, x, y, z, a, 0);
                        gather_f(p, fb, x, y, z, b, 0);
                        for (int i = 0; i < Q; i++) {
                            rr += a[i];
                            rb += b[i];
                        }
                        phi[cell_index(p, x, y, z)] = (rr - rb) / (rr + rb);
                    }
            /* Pass 2: single-phase CM collision of the total populations with
             * h_eq, perturbation, recolouring (Omega = Omega3[Omega1 + Omega2]). */
#pragma omp parallel for schedule(static) reduction(| : err)
            for (int z = 0; z < nz; z++)
                for (int y = 0; y < ny; y++)
                    for (int x = 0; x < nx; x++) {
                        long c = cell_index(p, x, y, z);
                        double a[Q], b[Q], ft[Q], fs[Q], grad[3];
                        gather_f(p, fr, x, y, z, a, 0);
                        gather_f(p, fb, x, y, z, b, 0);
                        double rr = 0, rb = 0;
                        for (int i = 0; i < Q; i++) {
                            ft[i] = a[i] + b[i];
                            rr += a[i];
                            rb += b[i];
                        }
                        node_state st;
                        node_macro(p, ft, NULL, &st);
                        double alpha = (rr * p->alpha_r + rb * p->alpha_b) / st.rho;
                        err |= collide(p, ft, &st, 1, alpha, fs) != 0;
                        cgm_gradient(p, phi, x, y, z, grad);
                        orc_cgm_perturb(grad, p->A, fs);
                        orc_cgm_recolour(fs, grad, rr, rb, alpha, p->beta, frtmp + c * Q, fbtmp + c * Q);
                    }
            memcpy(fr, frtmp, sizeof(double) * n * Q);
            memcpy(fb, fbtmp, sizeof(double) * n * Q);
            continue;
        }
        if (p->physics == 3) sc_pseudopotential(p, f, phi);
#pragma omp parallel for schedule(static) reduction(| : err)
        for (int z = 0; z < nz; z++)
            for (int y = 0; y < ny; y++)
                for (int x = 0; x < nx; x++) {
                    long c = cell_index(p, x, y, z);
                    double fin[Q], gin[21];
                    node_state st;
                    gather_f(p, f, x, y, z, fin, 1);
                    if (p->physics == 3) {
                        node_macro_sc(p, fin, NULL, phi, x, y, z, &st);
                        err |= collide(p, fin, &st, 0, 0.0, ftmp + c * Q) != 0;
                        continue;
                    }
                    if (p->physics == 1) gather_g(p, g, x, y, z, gin);
                    node_macro(p, fin, p->physics == 1 ? gin : NULL, &st);
                    err |= collide(p, fin, &st, 0, 0.0, ftmp + c * Q) != 0;
                    if (p->physics == 1) {
                        /* Magnetic BGK toward g_eq(u, b) with the corrected u. */
                        double geq[21];
                        orc_geq(st.u[0], st.u[1], st.u[2], st.b[0], st.b[1], st.b[2], geq);
                        for (int k = 0; k < 21; k++) gtmp[c * 21 + k] = gin[k] - (gin[k] - geq[k]) / p->tau_m;
                    }
                }
        memcpy(f, ftmp, sizeof(double) * n * Q);
        if (p->physics == 1) memcpy(g, gtmp, sizeof(double) * n * 21);
    }
    return err ? -1 : 0;
}

/* Macroscopic fields of the current state: moments of the gathered
 * populations (rho, u with +F/2), the order parameter (CGM) and b (MHD). */
int orc_fields(const orc_params *p, const double *f, const double *g, const double *fr, const double *fb, double *rho,
               double *u, double *phase, double *B)
{
    int nx = p->nx, ny = p->ny, nz = p->nz;
    long n = (long)nx * ny * nz;
    double *psi = NULL;
    if (p->physics == 3) {
        psi = (double *)malloc(sizeof(double) * n);
        if (!psi) return -1;
        sc_pseudopotential(p, f, psi);
    }
#pragma omp parallel for schedule(static)
    for (int z = 0; z < nz; z++)
        for (int y = 0; y < ny; y++)
            for (int x = 0; x < nx; x++) {
                long c = cell_index(p, x, y, z);
                double fin[Q], gin[21];
                node_state st;
                if (p->physics == 2) {
                    double a[Q], b[Q], rr = 0, rb = 0;
                    gather_f(p, fr, x, y, z, a, 0);
                    gather_f(p, fb, x, y, z, b, 0);
                    for (int i = 0; i < Q; i++) {
                        fin[i] = a[i] + b[i];
                        rr += a[i];
                        rb += b[i];
                    }
                    if (phase) phase[c] = (rr - rb) / (rr + rb);
                    node_macro(p, fin, NULL, &st);
                } else if (p->physics == 3) {
                    gather_f(p, f, x, y, z, fin, 1);
                    node_macro_sc(p, fin, NULL, psi, x, y, z, &st);
                    if (phase) phase[c] = psi[c];
                } else {
                    gather_f(p, f, x, y, z, fin, 1);
                    if (p->physics == 1) gather_g(p, g, x, y, z, gin);
                    node_macro(p, fin, p->physics == 1 ? gin : NULL, &st);
                    if (B) {
                        B[c] = st.b[0];
                        B[n + c] = st.b[1];
                        B[2 * n + c] = st.b[2];
                    }
                }
                if (rho) rho[c] = st.rho;
                if (u) {
                    u[c] = st.u[0];
                    u[n + c] = st.u[1];
                    u[2 * n + c] = st.u[2];
                }
            }
    free(psi);
    return 0;
}
