/*
 * FP64 CPU oracle for one implicit flux-limited-diffusion (FLD) radiation step,
 * written from Chen & Bai, "Guangqi" (arXiv 2602.12545), Sec. 3.2.
 *
 * TEST INFRASTRUCTURE ONLY: the slow, plain reference the CUDA path is checked
 * against.  Only the tests, the smoke check and the benchmark's CPU-baseline leg
 * may load it.  It shares nothing with the CUDA library.
 *
 * What it computes (Sec. 3.2.1):
 *   - the radiation / gas-energy sub-system, Eqs. radtran1-2, discretised by
 *     backward Euler, with (T^{n+1})^4 ~ 4 T^3 T^{n+1} - 3 T^4 (Sec. 3.2.1);
 *   - FLD flux F = -D grad E, D = c lambda(R) / (kappa_R rho) (Sec. 2, Eq. limiter,
 *     Eq. reducer), face values per Eq. diffcoeff;
 *   - the coefficients phi_1..phi_11, psi_5, psi_6, psi_11 (Eqs. phi1-psi7) with
 *     alpha = dt / (x_{m} - x_{k}) between volume centres (Eq. alpha) and the
 *     geometric factor g = dS / dV (Eq. fldg);
 *   - the coupled 2 N1 N2 linear system, Eqs. linearsys1-2.  T is eliminated exactly
 *     from the local psi row, leaving an N1 N2 symmetric positive-definite system in E
 *     that is solved directly (banded Gaussian elimination with partial pivoting) or by
 *     Jacobi-preconditioned conjugate gradients.  The paper-literal coupled system is
 *     also assembled and solvable by banded elimination, as a cross-check: in FP64 it
 *     loses all accuracy once beta_P >> 1 (phi_5 = 1 + ... + beta_P), so it is only
 *     compared where the coupling is moderate;
 *   - T^{n+1} back-substituted from the psi row, e_g^{n+1} = e_g^n + C_V (T^{n+1} - T^n).
 *   - the explicit advection source S_adv of Eq. adv (face mass flux times the upwind
 *     e_r = E / rho, times g = dS / dV), which enters phi_11 as S_adv dt; S_g = 0.
 *
 * Readings where the paper is silent or inconsistent (each one is a named choice):
 *   - D > 0 (Eq. diffcoeff prints a minus sign; only D > 0 makes phi_5 diagonally
 *     dominant as phi_5 = 1 - phi_1 - phi_3 - phi_7 - phi_9 + beta_P requires).
 *   - Signs of the exchange term follow the phi / psi coefficients: radiation loses
 *     dt G0, gas gains dt G0 (Eqs. radtran1-2 print the opposite sign).
 *   - Face sigma and face E: linear interpolation in the normal coordinate between
 *     the two volume centres (an arithmetic mean on uniform grids).
 *   - R at a face uses the normal one-sided difference |E_m - E_k| / d only.
 *   - Opacities at T_g^n, frozen over the step; kappa_e = kappa_P (Sec. 2).
 *   - Limiter 0 is the Levermore-Pomraning rational form (2+R)/(6+3R+R^2);
 *     1 is Minerbo (Eq. limiter); 2 is lambda = 1/3 (no limiting).
 *   - Milne boundary (Eq. milne) on a face at half-cell distance h from the centre:
 *     E_b = k/(1+k) E_k with k = 2/(3 sigma_k h); then |grad E|/(sigma E_b) = 3/2 so
 *     lambda_b = lambda(3/2) and D_b = c lambda_b / sigma_k; the face flux
 *     D_b (E_k - E_b)/h acts like a face to a zero-energy ghost at distance h (1+k).
 *   - Reflecting boundary: no flux through the face.
 *   - Eq. adv at a boundary face: the upwind e_r is that of the face's one cell (a
 *     zero-gradient ghost), whichever way the given mass flux points.
 *   - Non-linear C_V (Sec. 3.2.1 computes C_V per cell before the coefficients): with a
 *     table u(T) (piecewise linear), T^n inverts u = e_g / rho on the segment that holds
 *     it and C_V = rho du/dT of that segment; e_g^{n+1} = e_g^n + C_V (T^{n+1} - T^n).
 *   - Spherical-polar (r, theta), axisymmetric, the common factor 2 pi dropped:
 *     V = (r+^3 - r-^3)/3 (cos th- - cos th+), A_r = r^2 (cos th- - cos th+),
 *     A_th = sin th (r+^2 - r-^2)/2; volume centres r_c = int r dV / int dV and
 *     th_c = int th dV / int dV; the distance between theta-neighbours is r_c dth_c.
 */
#include "gq_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* CGS constants, written out for the oracle alone */
static const double C_LIGHT = 2.99792458e10;          /* cm / s */
static const double K_BOLTZ = 1.380649e-16;           /* erg / K */
static const double SIGMA_SB = 5.670374419e-5;        /* erg / (cm^2 s K^4) */
static const double AMU = 1.66053906660e-24;          /* g */
static const double M_HYDROGEN_U = 1.00782503207;     /* hydrogen atom mass in u */

double orc_const_c(void) { return C_LIGHT; }
double orc_const_aR(void) { return 4.0 * SIGMA_SB / C_LIGHT; }
double orc_const_kB(void) { return K_BOLTZ; }
double orc_const_mH(void) { return M_HYDROGEN_U * AMU; }

/* ------------------------------------------------------------------------- */
/* flux limiter lambda(R) (Sec. 2)                                             */
/* ------------------------------------------------------------------------- */
double orc_limiter(int kind, double R)
{
    if (kind == 2) return 1.0 / 3.0;
    if (kind == 1) {                       /* Minerbo, Eq. limiter */
        if (R <= 1.5) return 2.0 / (3.0 + sqrt(9.0 + 12.0 * R * R));
        return 1.0 / (1.0 + R + sqrt(1.0 + 2.0 * R));
    }
    return (2.0 + R) / (6.0 + 3.0 * R + R * R);   /* Levermore-Pomraning, rational form */
}

/* ------------------------------------------------------------------------- */
/* geometry: volumes, face areas, volume centres                               */
/* ------------------------------------------------------------------------- */
int orc_geometry(const orc_problem *P, double *V, double *Ax, double *Ay, double *xc, double *yc)
{
    const int nx = P->nx, ny = P->ny;
    if (nx < 1 || ny < 1) return -1;
    if (P->coord == 0) {
        for (int i = 0; i < nx; i++) xc[i] = 0.5 * (P->xf[i] + P->xf[i + 1]);
        for (int j = 0; j < ny; j++) yc[j] = 0.5 * (P->yf[j] + P->yf[j + 1]);
        for (int j = 0; j < ny; j++)
            for (int i = 0; i < nx; i++)
                V[j * nx + i] = (P->xf[i + 1] - P->xf[i]) * (P->yf[j + 1] - P->yf[j]);
        for (int j = 0; j < ny; j++)
            for (int i = 0; i <= nx; i++)
                Ax[j * (nx + 1) + i] = P->yf[j + 1] - P->yf[j];
        for (int j = 0; j <= ny; j++)
            for (int i = 0; i < nx; i++)
                Ay[j * nx + i] = P->xf[i + 1] - P->xf[i];
    } else {
        /* r: int r^2 dr = (r+^3 - r-^3)/3, written as (r+ - r-)(r+^2 + r+ r- + r-^2)/3;
         * r_c = int r^3 dr / int r^2 dr = (3/4)(r+^4 - r-^4)/(r+^3 - r-^3). */
        for (int i = 0; i < nx; i++) {
            double a = P->xf[i], b = P->xf[i + 1];
            xc[i] = 0.75 * (a + b) * (a * a + b * b) / (a * a + a * b + b * b);
        }
        /* theta: int sin = cos th- - cos th+ = 2 sin m sin(h/2) with m the mid-angle and
         * h the width; int th sin = [sin th - th cos th], which over the cell equals
         * 2 sin(h/2) [ m sin m + cos m (1 - (h/2) cot(h/2)) ]; so
         * th_c = m + cot(m) (1 - (h/2) cot(h/2)).  For small h/2 the bracket uses its
         * Taylor series x^2/3 + x^4/45 + 2 x^6/945 + x^8/4725 (x = h/2). */
        for (int j = 0; j < ny; j++) {
            double a = P->yf[j], b = P->yf[j + 1];
            double m = 0.5 * (a + b), x = 0.5 * (b - a);
            double bracket;
            if (x < 1e-2) {
                double x2 = x * x;
                bracket = x2 / 3.0 + x2 * x2 / 45.0 + 2.0 * x2 * x2 * x2 / 945.0 + x2 * x2 * x2 * x2 / 4725.0;
            } else {
                bracket = 1.0 - x * cos(x) / sin(x);
            }
            yc[j] = m + cos(m) / sin(m) * bracket;
        }
        for (int j = 0; j < ny; j++) {
            double a = P->yf[j], b = P->yf[j + 1];
            double dcos = 2.0 * sin(0.5 * (a + b)) * sin(0.5 * (b - a));
            for (int i = 0; i < nx; i++) {
                double r0 = P->xf[i], r1 = P->xf[i + 1];
                V[j * nx + i] = (r1 - r0) * (r1 * r1 + r1 * r0 + r0 * r0) / 3.0 * dcos;
            }
            for (int i = 0; i <= nx; i++) {
                double r = P->xf[i];
                Ax[j * (nx + 1) + i] = r * r * dcos;
            }
        }
        for (int j = 0; j <= ny; j++) {
            double s = sin(P->yf[j]);
            if (j == 0 && P->yf[0] == 0.0) s = 0.0;
            for (int i = 0; i < nx; i++) {
                double r0 = P->xf[i], r1 = P->xf[i + 1];
                Ay[j * nx + i] = s * (r1 - r0) * (r1 + r0) / 2.0;
            }
        }
    }
    if (P->V_in) memcpy(V, P->V_in, sizeof(double) * nx * ny);
    if (P->Ax_in) memcpy(Ax, P->Ax_in, sizeof(double) * ny * (nx + 1));
    if (P->Ay_in) memcpy(Ay, P->Ay_in, sizeof(double) * (ny + 1) * nx);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* per-cell and per-face quantities of the step                                */
/* ------------------------------------------------------------------------- */
typedef struct {
    int nx, ny, N;
    double *V, *Ax, *Ay, *xc, *yc;
    double *CV, *T, *sig, *betaP, *betaE;
    /* face weights: alpha * A * D = dt A D / d (per face, both neighbours use it) */
    double *wx, *wy;      /* [ny][nx+1], [ny+1][nx]; boundary entries: Milne ghost weights */
    double *Dx, *Dy, *Rx, *Ry, *dx, *dy;   /* diagnostics: D, R, distance used */
} orc_work;

static void work_free(orc_work *W)
{
    free(W->V); free(W->Ax); free(W->Ay); free(W->xc); free(W->yc);
    free(W->CV); free(W->T); free(W->sig); free(W->betaP); free(W->betaE);
    free(W->wx); free(W->wy); free(W->Dx); free(W->Dy); free(W->Rx); free(W->Ry);
    free(W->dx); free(W->dy);
}

static double opacity(const double k[4], double rho, double T)
{
    if (k[1] == 0.0) return k[0];
    return k[0] + k[1] * pow(rho, k[2]) * pow(T, k[3]);
}

static int work_build(const orc_problem *P, orc_work *W)
{
    const int nx = P->nx, ny = P->ny, N = nx * ny;
    memset(W, 0, sizeof(*W));
    W->nx = nx; W->ny = ny; W->N = N;
    W->V = calloc(N, sizeof(double));
    W->Ax = calloc((size_t)ny * (nx + 1), sizeof(double));
    W->Ay = calloc((size_t)(ny + 1) * nx, sizeof(double));
    W->xc = calloc(nx, sizeof(double));
    W->yc = calloc(ny, sizeof(double));
    W->CV = calloc(N, sizeof(double)); W->T = calloc(N, sizeof(double));
    W->sig = calloc(N, sizeof(double)); W->betaP = calloc(N, sizeof(double));
    W->betaE = calloc(N, sizeof(double));
    W->wx = calloc((size_t)ny * (nx + 1), sizeof(double));
    W->wy = calloc((size_t)(ny + 1) * nx, sizeof(double));
    W->Dx = calloc((size_t)ny * (nx + 1), sizeof(double));
    W->Dy = calloc((size_t)(ny + 1) * nx, sizeof(double));
    W->Rx = calloc((size_t)ny * (nx + 1), sizeof(double));
    W->Ry = calloc((size_t)(ny + 1) * nx, sizeof(double));
    W->dx = calloc((size_t)ny * (nx + 1), sizeof(double));
    W->dy = calloc((size_t)(ny + 1) * nx, sizeof(double));
    if (!W->V || !W->Ax || !W->Ay || !W->xc || !W->yc || !W->CV || !W->T || !W->sig ||
        !W->betaP || !W->betaE || !W->wx || !W->wy || !W->Dx || !W->Dy || !W->Rx || !W->Ry ||
        !W->dx || !W->dy) {
        work_free(W);
        return -2;
    }
    if (orc_geometry(P, W->V, W->Ax, W->Ay, W->xc, W->yc)) { work_free(W); return -1; }

    const double c = C_LIGHT;
    const double mH = orc_const_mH();
    /* cells: ideal-gas C_V = rho k_B / ((gamma-1) mu m_H) and T = e_g / C_V, or the table's
     * T(u) and C_V = rho du/dT on the segment holding u = e_g / rho; opacities at T^n */
    if (P->eos_n == 1 || P->eos_n < 0) { work_free(W); return -1; }
    for (int k = 0; k < N; k++) {
        double rho = P->rho[k];
        if (P->eos_n >= 2) {
            double u = P->eg[k] / rho;
            int s = 0;                          /* segment [s, s+1]: the last with u_s <= u */
            while (s + 2 < P->eos_n && P->eos_u[s + 1] <= u) s++;
            double slope = (P->eos_u[s + 1] - P->eos_u[s]) / (P->eos_T[s + 1] - P->eos_T[s]);
            W->T[k] = P->eos_T[s] + (u - P->eos_u[s]) / slope;
            W->CV[k] = rho * slope;
        } else {
            W->CV[k] = rho * K_BOLTZ / ((P->gamma - 1.0) * P->mu * mH);
            W->T[k] = P->eg[k] / W->CV[k];
        }
        double kR = opacity(P->kR, rho, W->T[k]);
        double kP = opacity(P->kP, rho, W->T[k]);
        W->sig[k] = kR * rho;
        W->betaP[k] = kP * rho * c * P->dt;     /* beta_P = kappa_P rho c dt */
        W->betaE[k] = W->betaP[k];             /* kappa_e = kappa_P */
    }

    /* interior x-faces: face i (1..nx-1) between cells (i-1, j) and (i, j) */
    for (int j = 0; j < ny; j++) {
        for (int i = 1; i < nx; i++) {
            int k = j * nx + i - 1, m = j * nx + i, f = j * (nx + 1) + i;
            double xk = W->xc[i - 1], xm = W->xc[i];
            double d = xm - xk;
            double th = (P->xf[i] - xk) / d;
            double sf = W->sig[k] + th * (W->sig[m] - W->sig[k]);
            double Ef = P->E[k] + th * (P->E[m] - P->E[k]);
            double R = fabs(P->E[m] - P->E[k]) / (d * sf * Ef);
            double D = c * orc_limiter(P->limiter, R) / sf;
            W->Rx[f] = R; W->Dx[f] = D; W->dx[f] = d;
            W->wx[f] = P->dt * W->Ax[f] * D / d;
        }
    }
    /* interior y-faces: face j (1..ny-1) between cells (i, j-1) and (i, j) */
    for (int j = 1; j < ny; j++) {
        for (int i = 0; i < nx; i++) {
            int k = (j - 1) * nx + i, m = j * nx + i, f = j * nx + i;
            double yk = W->yc[j - 1], ym = W->yc[j];
            double metric = (P->coord == 1) ? W->xc[i] : 1.0;
            double d = metric * (ym - yk);
            double th = (P->yf[j] - yk) / (ym - yk);
            double sf = W->sig[k] + th * (W->sig[m] - W->sig[k]);
            double Ef = P->E[k] + th * (P->E[m] - P->E[k]);
            double R = fabs(P->E[m] - P->E[k]) / (d * sf * Ef);
            double D = c * orc_limiter(P->limiter, R) / sf;
            W->Ry[f] = R; W->Dy[f] = D; W->dy[f] = d;
            W->wy[f] = P->dt * W->Ay[f] * D / d;
        }
    }
    /* Milne boundary faces: ghost weight dt A_b D_b / (h (1 + k)) */
    for (int side = 0; side < 4; side++) {
        if (P->bc[side] != 1) continue;
        if (side < 2) {
            int i = side == 0 ? 0 : nx;            /* face index */
            int ic = side == 0 ? 0 : nx - 1;       /* adjacent cell column */
            double h = fabs(P->xf[i] - W->xc[ic]);
            for (int j = 0; j < ny; j++) {
                int k = j * nx + ic, f = j * (nx + 1) + i;
                double s = W->sig[k];
                double kk = 2.0 / (3.0 * s * h);
                double D = c * orc_limiter(P->limiter, 1.5) / s;
                W->Rx[f] = 1.5; W->Dx[f] = D; W->dx[f] = h * (1.0 + kk);
                W->wx[f] = P->dt * W->Ax[f] * D / (h * (1.0 + kk));
            }
        } else {
            int j = side == 2 ? 0 : ny;
            int jc = side == 2 ? 0 : ny - 1;
            for (int i = 0; i < nx; i++) {
                double metric = (P->coord == 1) ? W->xc[i] : 1.0;
                double h = metric * fabs(P->yf[j] - W->yc[jc]);
                int k = jc * nx + i, f = j * nx + i;
                double s = W->sig[k];
                double kk = 2.0 / (3.0 * s * h);
                double D = c * orc_limiter(P->limiter, 1.5) / s;
                W->Ry[f] = 1.5; W->Dy[f] = D; W->dy[f] = h * (1.0 + kk);
                W->wy[f] = P->dt * W->Ay[f] * D / (h * (1.0 + kk));
            }
        }
    }
    /* frozen conductances (the paper's sub-cycle order keeps D from the start of the hydro
     * step and only updates alpha = dt / d): w = dt G, D = G d / A for the diagnostics and
     * the flux */
    if (P->Gx_in) {
        for (size_t f = 0; f < (size_t)ny * (nx + 1); f++) {
            W->wx[f] = P->dt * P->Gx_in[f];
            W->Dx[f] = W->Ax[f] > 0.0 && W->dx[f] > 0.0 ? P->Gx_in[f] * W->dx[f] / W->Ax[f] : 0.0;
        }
    }
    if (P->Gy_in) {
        for (size_t f = 0; f < (size_t)(ny + 1) * nx; f++) {
            W->wy[f] = P->dt * P->Gy_in[f];
            W->Dy[f] = W->Ay[f] > 0.0 && W->dy[f] > 0.0 ? P->Gy_in[f] * W->dy[f] / W->Ay[f] : 0.0;
        }
    }
    return 0;
}

int orc_faces(const orc_problem *P, double *Rx, double *Ry, double *Dx, double *Dy, double *wx, double *wy)
{
    orc_work W;
    int rc = work_build(P, &W);
    if (rc) return rc;
    size_t nfx = (size_t)P->ny * (P->nx + 1), nfy = (size_t)(P->ny + 1) * P->nx;
    if (Rx) memcpy(Rx, W.Rx, nfx * sizeof(double));
    if (Ry) memcpy(Ry, W.Ry, nfy * sizeof(double));
    if (Dx) memcpy(Dx, W.Dx, nfx * sizeof(double));
    if (Dy) memcpy(Dy, W.Dy, nfy * sizeof(double));
    if (wx) memcpy(wx, W.wx, nfx * sizeof(double));
    if (wy) memcpy(wy, W.wy, nfy * sizeof(double));
    work_free(&W);
    return 0;
}

/* The four faces of cell (i, j): neighbour cell index (or -1 for a boundary face)
 * and the face weight dt A D / d. */
static void cell_faces(const orc_problem *P, const orc_work *W, int i, int j, int nb[4], double w[4])
{
    const int nx = P->nx, ny = P->ny;
    nb[0] = i > 0 ? j * nx + i - 1 : -1;       w[0] = W->wx[j * (nx + 1) + i];
    nb[1] = i < nx - 1 ? j * nx + i + 1 : -1;  w[1] = W->wx[j * (nx + 1) + i + 1];
    nb[2] = j > 0 ? (j - 1) * nx + i : -1;     w[2] = W->wy[j * nx + i];
    nb[3] = j < ny - 1 ? (j + 1) * nx + i : -1; w[3] = W->wy[(j + 1) * nx + i];
}

/* Coefficients of Eqs. phi1-psi7 for cell k (per unit volume).  phi_nb[f] are the
 * neighbour coefficients -alpha g D (0 for boundary faces); phi_bnd is the Milne
 * ghost term, which has no unknown and so only enters phi_5. */
typedef struct { double phi_nb[4], phi5, phi6, phi11, psi5, psi6, psi11; } orc_coef;

static orc_coef cell_coef(const orc_problem *P, const orc_work *W, int i, int j)
{
    const double aR = orc_const_aR();
    int k = j * P->nx + i;
    int nb[4]; double w[4];
    cell_faces(P, W, i, j, nb, w);
    orc_coef C;
    double sum = 0.0;
    for (int f = 0; f < 4; f++) {
        /* alpha g D = (dt / d) (A / V) D = w / V */
        double agd = w[f] / W->V[k];
        C.phi_nb[f] = nb[f] >= 0 ? -agd : 0.0;
        sum += agd;     /* reflecting faces carry w = 0; Milne faces carry the ghost weight */
    }
    double T = W->T[k], T3 = T * T * T, T4 = T3 * T;
    C.phi5 = 1.0 + sum + W->betaP[k];
    C.phi6 = -4.0 * W->betaE[k] * aR * T3;
    C.phi11 = P->E[k] - 3.0 * W->betaE[k] * aR * T4 + (P->S_adv ? P->S_adv[k] : 0.0) * P->dt;   /* S_g = 0 */
    C.psi5 = -W->betaP[k];
    C.psi6 = W->CV[k] + 4.0 * W->betaE[k] * aR * T3;
    C.psi11 = W->CV[k] * T + 3.0 * W->betaE[k] * aR * T4;
    return C;
}

int orc_assemble_coupled(const orc_problem *P, int *rowptr, int *col, double *val, double *rhs)
{
    orc_work W;
    int rc = work_build(P, &W);
    if (rc) return rc;
    const int nx = P->nx, ny = P->ny;
    int nnz = 0;
    rowptr[0] = 0;
    for (int j = 0; j < ny; j++) {
        for (int i = 0; i < nx; i++) {
            int k = j * nx + i;
            int nb[4]; double w[4];
            cell_faces(P, &W, i, j, nb, w);
            orc_coef C = cell_coef(P, &W, i, j);
            /* E row: phi_1 E_{j-1} + phi_3 E_{i-1} + phi_5 E + phi_6 T + phi_7 E_{i+1} + phi_9 E_{j+1} */
            int order[4] = {2, 0, 1, 3};
            for (int t = 0; t < 2; t++) {          /* south, west (columns before 2k) */
                int f = order[t];
                if (nb[f] >= 0) { col[nnz] = 2 * nb[f]; val[nnz++] = C.phi_nb[f]; }
            }
            col[nnz] = 2 * k; val[nnz++] = C.phi5;
            col[nnz] = 2 * k + 1; val[nnz++] = C.phi6;
            for (int t = 2; t < 4; t++) {          /* east, north */
                int f = order[t];
                if (nb[f] >= 0) { col[nnz] = 2 * nb[f]; val[nnz++] = C.phi_nb[f]; }
            }
            rhs[2 * k] = C.phi11;
            rowptr[2 * k + 1] = nnz;
            /* T row: psi_5 E + psi_6 T = psi_11 */
            col[nnz] = 2 * k; val[nnz++] = C.psi5;
            col[nnz] = 2 * k + 1; val[nnz++] = C.psi6;
            rhs[2 * k + 1] = C.psi11;
            rowptr[2 * k + 2] = nnz;
        }
    }
    work_free(&W);
    return nnz;
}

int orc_assemble_reduced(const orc_problem *P, int *rowptr, int *col, double *val, double *rhs)
{
    orc_work W;
    int rc = work_build(P, &W);
    if (rc) return rc;
    const int nx = P->nx, ny = P->ny;
    int nnz = 0;
    rowptr[0] = 0;
    for (int j = 0; j < ny; j++) {
        for (int i = 0; i < nx; i++) {
            int k = j * nx + i;
            int nb[4]; double w[4];
            cell_faces(P, &W, i, j, nb, w);
            orc_coef C = cell_coef(P, &W, i, j);
            /* V_k (E row - (phi_6 / psi_6) T row): T eliminated exactly.
             * Diagonal: phi_5 - phi_6 psi_5 / psi_6 = 1 + sum(w)/V + beta_P - beta_P q / psi_6
             * with q = 4 beta_e a T^3 = psi_6 - C_V, i.e. 1 + sum(w)/V + beta_P C_V / psi_6.
             * Right-hand side: phi_11 - phi_6 psi_11 / psi_6 = E^n + beta_e a T^4 C_V / psi_6.
             * The oracle evaluates these right-hand forms: they are the same numbers, but
             * the printed forms subtract terms of size beta_P, which for stiff coupling
             * (q >> C_V) leaves no significant digits in FP64.
             * Off-diagonals are V_k phi_nb = -w_f, taken as the shared face weight so that
             * the matrix is exactly symmetric. */
            double Vk = W.V[k];
            double T = W.T[k], aT4 = orc_const_aR() * T * T * T * T;
            double diag = Vk * (1.0 + W.betaP[k] * W.CV[k] / C.psi6);
            for (int f = 0; f < 4; f++) diag += w[f];
            int order[4] = {2, 0, 1, 3};
            for (int t = 0; t < 2; t++) {
                int f = order[t];
                if (nb[f] >= 0) { col[nnz] = nb[f]; val[nnz++] = -w[f]; }
            }
            col[nnz] = k; val[nnz++] = diag;
            for (int t = 2; t < 4; t++) {
                int f = order[t];
                if (nb[f] >= 0) { col[nnz] = nb[f]; val[nnz++] = -w[f]; }
            }
            double Eadv = P->E[k] + (P->S_adv ? P->S_adv[k] : 0.0) * P->dt;
            rhs[k] = Vk * (Eadv + W.betaE[k] * aT4 * W.CV[k] / C.psi6);
            rowptr[k + 1] = nnz;
        }
    }
    work_free(&W);
    return nnz;
}

/* ------------------------------------------------------------------------- */
/* explicit advection source (Eq. adv)                                         */
/* ------------------------------------------------------------------------- */
int orc_adv_source(const orc_problem *P, const double *fx, const double *fy, double *S)
{
    const int nx = P->nx, ny = P->ny, N = nx * ny;
    double *V = malloc(sizeof(double) * N);
    double *Ax = malloc(sizeof(double) * ny * (nx + 1));
    double *Ay = malloc(sizeof(double) * (ny + 1) * nx);
    double *xc = malloc(sizeof(double) * nx), *yc = malloc(sizeof(double) * ny);
    int rc = (V && Ax && Ay && xc && yc) ? orc_geometry(P, V, Ax, Ay, xc, yc) : -2;
    if (rc == 0) {
        for (int j = 0; j < ny; j++) {
            for (int i = 0; i < nx; i++) {
                int k = j * nx + i;
                /* the four faces of cell k: -x, +x, -y, +y; the neighbour across each
                 * (-1 on a boundary) and the face's mass flux and area */
                int nb[4] = {i > 0 ? k - 1 : -1, i < nx - 1 ? k + 1 : -1,
                             j > 0 ? k - nx : -1, j < ny - 1 ? k + nx : -1};
                double f[4] = {fx[j * (nx + 1) + i], fx[j * (nx + 1) + i + 1], fy[j * nx + i], fy[(j + 1) * nx + i]};
                double A[4] = {Ax[j * (nx + 1) + i], Ax[j * (nx + 1) + i + 1], Ay[j * nx + i], Ay[(j + 1) * nx + i]};
                double s = 0.0;
                for (int t = 0; t < 4; t++) {
                    /* the flow enters through a lower face when f > 0 and through an
                     * upper face when f < 0; the upwind cell is then the neighbour */
                    int lower = (t % 2) == 0;
                    int in = lower ? f[t] > 0.0 : f[t] < 0.0;
                    int up = (in && nb[t] >= 0) ? nb[t] : k;
                    double er = P->E[up] / P->rho[up];
                    double g = A[t] / V[k];
                    /* lower faces add g f e_r, upper faces subtract it */
                    s += (lower ? 1.0 : -1.0) * g * f[t] * er;
                }
                S[k] = s;
            }
        }
    }
    free(V); free(Ax); free(Ay); free(xc); free(yc);
    return rc;
}

/* ------------------------------------------------------------------------- */
/* direct solver: banded Gaussian elimination with partial pivoting            */
/* ------------------------------------------------------------------------- */
int orc_band_solve(int n, const int *rowptr, const int *col, const double *val, const double *rhs, double *x)
{
    int kl = 0, ku = 0;
    for (int i = 0; i < n; i++)
        for (int p = rowptr[i]; p < rowptr[i + 1]; p++) {
            int d = col[p] - i;
            if (-d > kl) kl = -d;
            if (d > ku) ku = d;
        }
    const int width = 2 * kl + ku + 1;    /* room for the fill-in that row swaps create */
    if (n <= 0 || width <= 0) return -1;
    double *B = calloc((size_t)n * (size_t)width, sizeof(double));
    double *b = malloc(sizeof(double) * n);
    if (!B || !b) { free(B); free(b); return -2; }
#define AB(i, j) B[(size_t)(i) * width + ((j) - (i) + kl)]
    for (int i = 0; i < n; i++) {
        for (int p = rowptr[i]; p < rowptr[i + 1]; p++) AB(i, col[p]) += val[p];
        b[i] = rhs[i];
    }
    for (int k = 0; k < n; k++) {
        int last = k + kl < n - 1 ? k + kl : n - 1;
        int piv = k;
        double best = fabs(AB(k, k));
        for (int i = k + 1; i <= last; i++)
            if (fabs(AB(i, k)) > best) { best = fabs(AB(i, k)); piv = i; }
        if (best == 0.0) { free(B); free(b); return -3; }
        int jend = k + kl + ku < n - 1 ? k + kl + ku : n - 1;
        if (piv != k) {
            for (int j = k; j <= jend; j++) { double t = AB(k, j); AB(k, j) = AB(piv, j); AB(piv, j) = t; }
            double t = b[k]; b[k] = b[piv]; b[piv] = t;
        }
        for (int i = k + 1; i <= last; i++) {
            double l = AB(i, k) / AB(k, k);
            if (l == 0.0) continue;
            for (int j = k; j <= jend; j++) AB(i, j) -= l * AB(k, j);
            b[i] -= l * b[k];
        }
    }
    for (int i = n - 1; i >= 0; i--) {
        int jend = i + kl + ku < n - 1 ? i + kl + ku : n - 1;
        double s = b[i];
        for (int j = i + 1; j <= jend; j++) s -= AB(i, j) * x[j];
        x[i] = s / AB(i, i);
    }
#undef AB
    free(B); free(b);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* iterative solver: Jacobi-preconditioned conjugate gradients                 */
/* ------------------------------------------------------------------------- */
static void csr_mv(int n, const int *rowptr, const int *col, const double *val, const double *x, double *y)
{
    for (int i = 0; i < n; i++) {
        double s = 0.0;
        for (int p = rowptr[i]; p < rowptr[i + 1]; p++) s += val[p] * x[col[p]];
        y[i] = s;
    }
}

static double cellwise(int n, const double *r, const double *diag, const double *x)
{
    double m = 0.0;
    for (int i = 0; i < n; i++) {
        double c = fabs(r[i]) / (diag[i] * fabs(x[i]));
        if (!(c <= m)) m = c;      /* also propagates NaN */
    }
    return m;
}

int orc_pcg(int n, const int *rowptr, const int *col, const double *val, const double *rhs,
            double *x, double tol, int maxit, int *iters, double *crit)
{
    double *diag = malloc(sizeof(double) * n), *r = malloc(sizeof(double) * n);
    double *z = malloc(sizeof(double) * n), *p = malloc(sizeof(double) * n);
    double *q = malloc(sizeof(double) * n);
    if (!diag || !r || !z || !p || !q) { free(diag); free(r); free(z); free(p); free(q); return -2; }
    for (int i = 0; i < n; i++) {
        diag[i] = 0.0;
        for (int k = rowptr[i]; k < rowptr[i + 1]; k++) if (col[k] == i) diag[i] = val[k];
    }
    csr_mv(n, rowptr, col, val, x, q);
    double rho = 0.0;
    for (int i = 0; i < n; i++) { r[i] = rhs[i] - q[i]; z[i] = r[i] / diag[i]; p[i] = z[i]; rho += r[i] * z[i]; }
    int it = 0;
    double c = cellwise(n, r, diag, x);
    while (c > tol && it < maxit) {
        csr_mv(n, rowptr, col, val, p, q);
        double pq = 0.0;
        for (int i = 0; i < n; i++) pq += p[i] * q[i];
        double alpha = rho / pq;
        for (int i = 0; i < n; i++) { x[i] += alpha * p[i]; r[i] -= alpha * q[i]; }
        double rho_new = 0.0;
        for (int i = 0; i < n; i++) { z[i] = r[i] / diag[i]; rho_new += r[i] * z[i]; }
        double beta = rho_new / rho;
        for (int i = 0; i < n; i++) p[i] = z[i] + beta * p[i];
        rho = rho_new;
        it++;
        c = cellwise(n, r, diag, x);
    }
    /* report the criterion of the true residual b - A x */
    csr_mv(n, rowptr, col, val, x, q);
    for (int i = 0; i < n; i++) r[i] = rhs[i] - q[i];
    *crit = cellwise(n, r, diag, x);
    *iters = it;
    free(diag); free(r); free(z); free(p); free(q);
    return it < maxit || c <= tol ? 0 : 1;
}

/* ------------------------------------------------------------------------- */
/* one implicit step                                                           */
/* ------------------------------------------------------------------------- */
int orc_step(const orc_problem *P, int method, double tol, double *E_new, double *T_new,
             double *eg_new, double *info, double *Fx, double *Fy)
{
    const int nx = P->nx, ny = P->ny, N = nx * ny;
    orc_work W;
    int rc = work_build(P, &W);
    if (rc) return rc;
    int iters = 0;
    double crit = 0.0;
    int status = 0;

    if (method == 2) {
        /* paper-literal coupled system (Eqs. linearsys1-2), banded LU */
        int *rp = malloc(sizeof(int) * (2 * N + 1)), *cl = malloc(sizeof(int) * 8 * N);
        double *vl = malloc(sizeof(double) * 8 * N), *rhs = malloc(sizeof(double) * 2 * N);
        double *xs = malloc(sizeof(double) * 2 * N);
        if (!rp || !cl || !vl || !rhs || !xs) status = -2;
        else {
            orc_assemble_coupled(P, rp, cl, vl, rhs);
            status = orc_band_solve(2 * N, rp, cl, vl, rhs, xs);
            for (int k = 0; k < N; k++) { E_new[k] = xs[2 * k]; T_new[k] = xs[2 * k + 1]; }
        }
        free(rp); free(cl); free(vl); free(rhs); free(xs);
        if (status) { work_free(&W); return status; }
    } else {
        for (int k = 0; k < N; k++) E_new[k] = P->E[k];    /* initial guess E^n */
    }

    /* reduced system: solved by banded LU (method 0) or CG (method 1); for method 2 it
     * only reports the residual of the coupled solution's E */
    {
        int *rp = malloc(sizeof(int) * (N + 1)), *cl = malloc(sizeof(int) * 5 * N);
        double *vl = malloc(sizeof(double) * 5 * N), *rhs = malloc(sizeof(double) * N);
        double *ax = malloc(sizeof(double) * N);
        if (!rp || !cl || !vl || !rhs || !ax) {
            free(rp); free(cl); free(vl); free(rhs); free(ax); work_free(&W); return -2;
        }
        orc_assemble_reduced(P, rp, cl, vl, rhs);
        if (method == 0) status = orc_band_solve(N, rp, cl, vl, rhs, E_new);
        else if (method == 1) status = orc_pcg(N, rp, cl, vl, rhs, E_new, tol, 1000000, &iters, &crit);
        csr_mv(N, rp, cl, vl, E_new, ax);
        double rr = 0.0, bb = 0.0, cw = 0.0;
        for (int k = 0; k < N; k++) {
            double r = rhs[k] - ax[k];
            rr += r * r; bb += rhs[k] * rhs[k];
            double dg = 0.0;
            for (int p = rp[k]; p < rp[k + 1]; p++) if (cl[p] == k) dg = vl[p];
            double c = fabs(r) / (dg * fabs(E_new[k]));
            if (!(c <= cw)) cw = c;
        }
        if (method != 1) crit = cw;
        if (info) { info[1] = crit; info[2] = sqrt(rr) / sqrt(bb); }
        free(rp); free(cl); free(vl); free(rhs); free(ax);
        if (status < 0) { work_free(&W); return status; }
    }

    /* back-substitution from the psi row (CG path), new gas energy, energy sums */
    double e0 = 0.0, e1 = 0.0;
    for (int j = 0; j < ny; j++) {
        for (int i = 0; i < nx; i++) {
            int k = j * nx + i;
            orc_coef C = cell_coef(P, &W, i, j);
            /* T^{n+1} = (psi_11 - psi_5 E^{n+1}) / psi_6: all terms positive, no cancellation */
            if (method != 2) T_new[k] = (C.psi11 - C.psi5 * E_new[k]) / C.psi6;
            eg_new[k] = P->eg[k] + W.CV[k] * (T_new[k] - W.T[k]);
            e0 += W.V[k] * (P->E[k] + P->eg[k]);
            e1 += W.V[k] * (E_new[k] + eg_new[k]);
        }
    }
    if (info) { info[0] = iters; info[3] = e0; info[4] = e1; }

    /* post-step face flux D^n (E^{n+1}_k - E^{n+1}_m) / d, positive along +x / +y */
    if (Fx) {
        for (int j = 0; j < ny; j++)
            for (int i = 0; i <= nx; i++) {
                int f = j * (nx + 1) + i;
                double F = 0.0;
                if (i > 0 && i < nx) F = -W.Dx[f] * (E_new[j * nx + i] - E_new[j * nx + i - 1]) / W.dx[f];
                else if (i == 0 && P->bc[0] == 1) F = -W.Dx[f] * E_new[j * nx] / W.dx[f];
                else if (i == nx && P->bc[1] == 1) F = W.Dx[f] * E_new[j * nx + nx - 1] / W.dx[f];
                Fx[f] = F;
            }
    }
    if (Fy) {
        for (int j = 0; j <= ny; j++)
            for (int i = 0; i < nx; i++) {
                int f = j * nx + i;
                double F = 0.0;
                if (j > 0 && j < ny) F = -W.Dy[f] * (E_new[j * nx + i] - E_new[(j - 1) * nx + i]) / W.dy[f];
                else if (j == 0 && P->bc[2] == 1) F = -W.Dy[f] * E_new[i] / W.dy[f];
                else if (j == ny && P->bc[3] == 1) F = W.Dy[f] * E_new[(ny - 1) * nx + i] / W.dy[f];
                Fy[f] = F;
            }
    }
    work_free(&W);
    return status;
}
