/*
 * FP64 CPU oracle for one implicit FLD radiation step (Chen & Bai, Guangqi, Sec. 3.2).
 *
 * TEST INFRASTRUCTURE ONLY.  This is the slow, plain reference the CUDA path is
 * checked against.  Only the test suite, the smoke check and the benchmark's CPU
 * baseline leg may load it.  It shares no code, header, table or constant with the
 * CUDA library; every constant below is written out here independently.
 *
 * Layout: cell fields are row-major [ny][nx] (x fastest).  x-face arrays are
 * [ny][nx+1] (face i sits between cells i-1 and i), y-face arrays are [ny+1][nx].
 * Boundary sides are ordered -x, +x, -y, +y.
 */
#ifndef GQ_ORACLE_H
#define GQ_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    int nx, ny;
    int coord;                /* 0 Cartesian (x, y); 1 spherical-polar (r, theta), axisymmetric */
    const double *xf, *yf;    /* face coordinates, nx+1 and ny+1 */
    const double *V_in;       /* optional explicit cell volumes [ny][nx] (NULL: derive) */
    const double *Ax_in;      /* optional explicit x-face areas [ny][nx+1] (NULL: derive) */
    const double *Ay_in;      /* optional explicit y-face areas [ny+1][nx] (NULL: derive) */
    const double *rho, *eg, *E;   /* density, gas internal energy per volume, radiation energy */
    double kR[4];             /* Rosseland law kappa = k0 + k1 rho^a T^b : {k0, k1, a, b} */
    double kP[4];             /* Planck law, same form */
    double gamma, mu;         /* ideal-gas EoS */
    double dt;
    int bc[4];                /* 0 reflecting, 1 Milne outflow */
    int limiter;              /* 0 Levermore-Pomraning (rational), 1 Minerbo, 2 none (1/3) */
    const double *S_adv;      /* optional explicit radiation source [ny][nx] (NULL: none),
                                 erg cm^-3 s^-1: the S_adv of phi_11 (Eq. adv) */
    const double *Gx_in, *Gy_in;  /* optional frozen face conductances A D / d per face,
                                 [ny][nx+1] and [ny+1][nx] (NULL: formed from this state);
                                 given, every face weight is dt G (Milne faces included) */
    int eos_n;                /* tabulated EoS: 0 = ideal gas (gamma, mu); else eos_n >= 2 points */
    const double *eos_T, *eos_u;  /* increasing T (K) and specific internal energy u (erg/g);
                                 u(T) piecewise linear, extended linearly past both ends */
} orc_problem;

/* physical constants (CGS) */
double orc_const_c(void);
double orc_const_aR(void);
double orc_const_kB(void);
double orc_const_mH(void);

double orc_limiter(int kind, double R);

int orc_geometry(const orc_problem *P, double *V, double *Ax, double *Ay, double *xc, double *yc);

/* Face diagnostics at time level n: R, lambda, D, w = dt A D / d for every face
 * (0 on reflecting boundary faces; Milne faces hold their boundary values). */
int orc_faces(const orc_problem *P, double *Rx, double *Ry, double *Dx, double *Dy, double *wx, double *wy);

/* Paper-literal coupled system, 2N unknowns interleaved [E_k, T_k], one row per
 * equation exactly as the phi / psi coefficients define it (rows per unit volume). */
int orc_assemble_coupled(const orc_problem *P, int *rowptr, int *col, double *val, double *rhs);

/* Schur-reduced N x N system in E (T eliminated exactly), rows multiplied by V_k. */
int orc_assemble_reduced(const orc_problem *P, int *rowptr, int *col, double *val, double *rhs);

/* Banded Gaussian elimination with partial pivoting on a CSR matrix. */
int orc_band_solve(int n, const int *rowptr, const int *col, const double *val, const double *rhs, double *x);

/* Jacobi-preconditioned CG on a symmetric CSR matrix; stops when the cell-wise relative
 * residual max_k |r_k| / (A_kk |x_k|) <= tol.  x holds the initial guess on entry. */
int orc_pcg(int n, const int *rowptr, const int *col, const double *val, const double *rhs,
            double *x, double tol, int maxit, int *iters, double *crit);

/* Eq. adv: S_adv per cell from the face mass fluxes fx [ny][nx+1], fy [ny+1][nx]
 * (g cm^-2 s^-1, positive along +x / +y) and the upwind specific radiation energy
 * e_r = E / rho, with g = dS / dV (Eq. fldg).  A boundary face takes e_r of its one cell. */
int orc_adv_source(const orc_problem *P, const double *fx, const double *fy, double *S);

/* One implicit step.  method 0: banded LU on the reduced system; 1: CG on the reduced
 * system to the cell-wise tol; 2: banded LU on the paper-literal coupled system.  Outputs E^{n+1}, T^{n+1}, e_g^{n+1}.  info (may be NULL) receives
 * {iterations, cell-wise residual, paper 2-norm residual |b-Ax|/|b| of the reduced
 * system, energy before, energy after}.  Fx/Fy (may be NULL) receive the post-step
 * face flux D^n (E^{n+1}_m - E^{n+1}_k)/d with the sign of -D grad E. */
int orc_step(const orc_problem *P, int method, double tol, double *E_new, double *T_new,
             double *eg_new, double *info, double *Fx, double *Fy);

#ifdef __cplusplus
}
#endif
#endif
