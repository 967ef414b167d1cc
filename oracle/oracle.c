/*
 * FP64 sequential CPU oracle for the mesh loops -- TEST INFRASTRUCTURE.
 *
 * Only the test suite, the smoke check and the benchmark's CPU-baseline leg
 * load this file.  The GPU library never includes, links or calls it, and it
 * shares no code with the GPU library: every loop below is a plain
 * iteration over the from-set in the order the maps are given, written from
 * the definitions it cites.
 *
 * Paper: "Locality Optimized Unstructured Mesh Algorithms on GPUs"
 * (Sulyok, Balogh, Reguly, Mudalige, 2018).  The paper fixes the access
 * pattern of each loop (Sec. 3.1.1: res_calc reads 5 doubles and increments 4
 * on each of 2 cells and reads 2 doubles on each of 2 nodes; Sec. 3.1.4:
 * IntegrateStressForElems reads 3 doubles on each of 8 nodes and increments
 * 3 per node) and the semantics of an indirect increment (Sec. 1.1.1), but
 * prints no formula.  The formulas below are the readings this library
 * adopts, each a textbook definition:
 *
 *   res_calc   central flux with scalar dissipation for the 2D Euler
 *              equations (Sec. 3.1.1 names the discretisation).
 *   bres_calc  the same flux on a far-field boundary edge.
 *   adt_calc   a spectral-radius time-step measure over the cell's edges.
 *   update     q = q_old - res/adt, res = 0, sum of squared updates.
 *   hex_force  one-point trilinear hex8 element: stress force -sigma B_i
 *              plus Flanagan-Belytschko hourglass control.
 *   adjoint    reverse-mode derivative of res_calc in q and x (adt fixed).
 *   space_disc an increment-only edge loop with the access pattern of
 *              Volna's SpaceDiscretization (Sec. 3.1.2: per edge 7 floats
 *              and 1 integer read directly, 1 value read and 4 incremented
 *              on each of 2 cells): the flux through the edge, already
 *              given per edge, integrated over its length, plus a pressure
 *              term along the normal, scaled by each cell's inverse area.
 *   face_flux  a finite-volume face flux with the access pattern of
 *              miniAero's compute_face_flux (Sec. 3.1.5: per face 12 doubles
 *              read directly, 28 read and 5 incremented on each of 2 cells):
 *              limited linear reconstruction to the face, the Rusanov
 *              (local Lax-Friedrichs) flux of the 3D Euler equations, and a
 *              Newtonian viscous and heat flux from face gradients.
 *   getacc     an increment-only cell loop with the access pattern of
 *              BookLeaf's getacc_scatter (Sec. 3.1.3: 17 doubles read
 *              directly per cell, 4 incremented on each of 4 nodes): the
 *              cell's corner mass, density-weighted corner area and corner
 *              forces gathered onto the nodes.
 *
 * All arrays are array-of-structures in the caller's numbering:
 * x[node][2], q[cell][4], adt[cell], res[cell][4], hex x/v[node][3],
 * sig[elem][3], f[node][3], vol[elem].  Maps are int32 row-major n x arity.
 * Increments are "+=": callers zero outputs first.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

/* ---------------------------------------------------------------- flux */

/* Normal flux F(q).n of the 2D Euler equations for conserved q = (rho, rho u,
 * rho v, E), pressure p = (gam-1)(E - |rho u|^2 / (2 rho)) and normal
 * velocity V = (rho u . n) / rho:
 *   F.n = (rho V, rho u V + p n_x, rho v V + p n_y, (E + p) V).          */
static void euler_flux(const double *q, double nx, double ny, double gam, double *F)
{
    double rho = q[0], ru = q[1], rv = q[2], E = q[3];
    double p = (gam - 1.0) * (E - 0.5 * (ru * ru + rv * rv) / rho);
    double V = (ru * nx + rv * ny) / rho;
    F[0] = rho * V;
    F[1] = ru * V + p * nx;
    F[2] = rv * V + p * ny;
    F[3] = (E + p) * V;
}

/* Interior-edge flux f (Sec. 3.1.1 res_calc):  with n = (y_a - y_b,
 * -(x_a - x_b)) for edge nodes (a, b),
 *   f = (F(q1).n + F(q2).n) / 2 + mu (q1 - q2),  mu = eps (adt1 + adt2) / 2. */
void oracle_edge_flux(const double *xa, const double *xb, const double *q1, const double *q2,
                      double adt1, double adt2, double gam, double eps, double *f)
{
    double nx = xa[1] - xb[1];
    double ny = -(xa[0] - xb[0]);
    double F1[4], F2[4];
    euler_flux(q1, nx, ny, gam, F1);
    euler_flux(q2, nx, ny, gam, F2);
    double mu = 0.5 * (adt1 + adt2) * eps;
    for (int k = 0; k < 4; ++k)
        f[k] = 0.5 * (F1[k] + F2[k]) + mu * (q1[k] - q2[k]);
}

/* res_calc: loop over interior edges, res[c1] += f, res[c2] -= f
 * (indirect increment, Sec. 1.1.1 and Algorithm 1's semantics). */
void oracle_res_calc(int64_t nedge, const int32_t *edge2node, const int32_t *edge2cell,
                     const double *x, const double *q, const double *adt, double *res,
                     double gam, double eps)
{
    for (int64_t e = 0; e < nedge; ++e) {
        int32_t a = edge2node[2 * e], b = edge2node[2 * e + 1];
        int32_t c1 = edge2cell[2 * e], c2 = edge2cell[2 * e + 1];
        double f[4];
        oracle_edge_flux(x + 2 * a, x + 2 * b, q + 4 * c1, q + 4 * c2, adt[c1], adt[c2], gam, eps, f);
        for (int k = 0; k < 4; ++k) {
            res[4 * c1 + k] += f[k];
            res[4 * c2 + k] -= f[k];
        }
    }
}

/* bres_calc (far-field boundary, Sec. 3.1.1 names the loop): with the
 * boundary state q_b = (q_c + q_inf)/2,
 *   f = F(q_b).n + eps adt_c (q_c - q_inf),  res[c] += f.               */
void oracle_bres_calc(int64_t nbedge, const int32_t *bedge2node, const int32_t *bedge2cell,
                      const double *x, const double *q, const double *adt, double *res,
                      const double *qinf, double gam, double eps)
{
    for (int64_t e = 0; e < nbedge; ++e) {
        int32_t a = bedge2node[2 * e], b = bedge2node[2 * e + 1];
        int32_t c = bedge2cell[e];
        double nx = x[2 * a + 1] - x[2 * b + 1];
        double ny = -(x[2 * a] - x[2 * b]);
        double qb[4], F[4];
        for (int k = 0; k < 4; ++k)
            qb[k] = 0.5 * (q[4 * c + k] + qinf[k]);
        euler_flux(qb, nx, ny, gam, F);
        for (int k = 0; k < 4; ++k)
            res[4 * c + k] += F[k] + eps * adt[c] * (q[4 * c + k] - qinf[k]);
    }
}

/* adt_calc: for each cell, sum over its 4 edges (corners in cyclic order)
 * of (|u dy - v dx| + c sqrt(dx^2 + dy^2)) / cfl, with u = rho u / rho,
 * v = rho v / rho and sound speed c = sqrt(gam p / rho).                 */
void oracle_adt_calc(int64_t ncell, const int32_t *cell2node, const double *x, const double *q,
                     double *adt, double gam, double cfl)
{
    for (int64_t c = 0; c < ncell; ++c) {
        const double *qc = q + 4 * c;
        double u = qc[1] / qc[0], v = qc[2] / qc[0];
        double p = (gam - 1.0) * (qc[3] - 0.5 * qc[0] * (u * u + v * v));
        double cs = sqrt(gam * p / qc[0]);
        double s = 0.0;
        for (int k = 0; k < 4; ++k) {
            int32_t n0 = cell2node[4 * c + k], n1 = cell2node[4 * c + (k + 1) % 4];
            double dx = x[2 * n1] - x[2 * n0], dy = x[2 * n1 + 1] - x[2 * n0 + 1];
            s += fabs(u * dy - v * dx) + cs * sqrt(dx * dx + dy * dy);
        }
        adt[c] = s / cfl;
    }
}

/* save_soln: q_old = q. */
void oracle_save_soln(int64_t ncell, const double *q, double *qold)
{
    memcpy(qold, q, (size_t)ncell * 4 * sizeof(double));
}

/* update: delta = res/adt, q = q_old - delta, res = 0, *rms_sum += sum delta^2. */
void oracle_update(int64_t ncell, const double *qold, double *q, double *res, const double *adt,
                   double *rms_sum)
{
    double s = 0.0;
    for (int64_t c = 0; c < ncell; ++c) {
        for (int k = 0; k < 4; ++k) {
            double d = res[4 * c + k] / adt[c];
            q[4 * c + k] = qold[4 * c + k] - d;
            res[4 * c + k] = 0.0;
            s += d * d;
        }
    }
    *rms_sum += s;
}

/* One time step: save_soln, then adt_calc, res_calc, bres_calc, update.
 * Returns the reported residual sqrt(sum delta^2 / ncell).  res must be 0
 * on entry (update leaves it 0).  adt and qold are scratch outputs.      */
double oracle_step(int64_t ncell, int64_t nedge, int64_t nbedge, const int32_t *cell2node,
                   const int32_t *edge2node, const int32_t *edge2cell, const int32_t *bedge2node,
                   const int32_t *bedge2cell, const double *x, double *q, double *qold, double *adt,
                   double *res, const double *qinf, double gam, double eps, double cfl)
{
    double rms = 0.0;
    oracle_save_soln(ncell, q, qold);
    oracle_adt_calc(ncell, cell2node, x, q, adt, gam, cfl);
    oracle_res_calc(nedge, edge2node, edge2cell, x, q, adt, res, gam, eps);
    oracle_bres_calc(nbedge, bedge2node, bedge2cell, x, q, adt, res, qinf, gam, eps);
    oracle_update(ncell, qold, q, res, adt, &rms);
    return sqrt(rms / (double)ncell);
}

/* --------------------------------------------------------- hex assembly */

/* Reference corners xi_i in {-1,+1}^3 of the trilinear hex8 element, in the
 * local order of the elem->node map. */
static const double XI[8][3] = {{-1, -1, -1}, {1, -1, -1}, {1, 1, -1}, {-1, 1, -1},
                                {-1, -1, 1},  {1, -1, 1},  {1, 1, 1},  {-1, 1, 1}};

/* Per-element nodal forces of the hex8 element with one-point quadrature
 * (Flanagan and Belytschko, IJNME 17, 1981):
 *   J   = 1/8 sum_i x_i (x) xi_i          (J_ab = dx_a / dxi_b at the centre)
 *   V   = 8 det J                         (written to vol)
 *   B_i = cof(J) xi_i,  cof(J) = det(J) J^{-T}
 *   f_i^s  = -diag(sxx, syy, szz) B_i
 *   Gamma_{k,i} = (eta zeta, xi zeta, xi eta, xi eta zeta)_i, k = 1..4
 *   g_{k,i} = Gamma_{k,i} - (1/V) (sum_j Gamma_{k,j} x_j) . B_i
 *   f_i^hg = -kappa sum_k g_{k,i} (sum_j g_{k,j} v_j)
 * and f[node_i] += f_i^s + f_i^hg.                                       */
void oracle_hex_element(const double xe[8][3], const double ve[8][3], const double *sig,
                        double kappa, double fe[8][3], double *vol)
{
    double J[3][3] = {{0}};
    for (int i = 0; i < 8; ++i)
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b)
                J[a][b] += 0.125 * xe[i][a] * XI[i][b];
    double C[3][3]; /* cofactor matrix: C_ab = (-1)^(a+b) minor_ab */
    C[0][0] = J[1][1] * J[2][2] - J[1][2] * J[2][1];
    C[0][1] = -(J[1][0] * J[2][2] - J[1][2] * J[2][0]);
    C[0][2] = J[1][0] * J[2][1] - J[1][1] * J[2][0];
    C[1][0] = -(J[0][1] * J[2][2] - J[0][2] * J[2][1]);
    C[1][1] = J[0][0] * J[2][2] - J[0][2] * J[2][0];
    C[1][2] = -(J[0][0] * J[2][1] - J[0][1] * J[2][0]);
    C[2][0] = J[0][1] * J[1][2] - J[0][2] * J[1][1];
    C[2][1] = -(J[0][0] * J[1][2] - J[0][2] * J[1][0]);
    C[2][2] = J[0][0] * J[1][1] - J[0][1] * J[1][0];
    double det = J[0][0] * C[0][0] + J[0][1] * C[0][1] + J[0][2] * C[0][2];
    double V = 8.0 * det;
    double B[8][3];
    for (int i = 0; i < 8; ++i)
        for (int a = 0; a < 3; ++a)
            B[i][a] = C[a][0] * XI[i][0] + C[a][1] * XI[i][1] + C[a][2] * XI[i][2];
    for (int i = 0; i < 8; ++i)
        for (int a = 0; a < 3; ++a)
            fe[i][a] = -sig[a] * B[i][a];
    double G[4][8];
    for (int i = 0; i < 8; ++i) {
        G[0][i] = XI[i][1] * XI[i][2];
        G[1][i] = XI[i][0] * XI[i][2];
        G[2][i] = XI[i][0] * XI[i][1];
        G[3][i] = XI[i][0] * XI[i][1] * XI[i][2];
    }
    for (int k = 0; k < 4; ++k) {
        double hk[3] = {0, 0, 0};
        for (int j = 0; j < 8; ++j)
            for (int a = 0; a < 3; ++a)
                hk[a] += G[k][j] * xe[j][a];
        double g[8];
        for (int i = 0; i < 8; ++i)
            g[i] = G[k][i] - (hk[0] * B[i][0] + hk[1] * B[i][1] + hk[2] * B[i][2]) / V;
        double qk[3] = {0, 0, 0};
        for (int j = 0; j < 8; ++j)
            for (int a = 0; a < 3; ++a)
                qk[a] += g[j] * ve[j][a];
        for (int i = 0; i < 8; ++i)
            for (int a = 0; a < 3; ++a)
                fe[i][a] -= kappa * g[i] * qk[a];
    }
    *vol = V;
}

/* Hex assembly loop (Sec. 3.1.4's IntegrateStressForElems access pattern):
 * gather x, v on 8 nodes, write vol directly, increment f on 8 nodes.    */
void oracle_hex_force(int64_t nelem, const int32_t *elem2node, const double *x, const double *v,
                      const double *sig, double *f, double *vol, double kappa)
{
    for (int64_t e = 0; e < nelem; ++e) {
        double xe[8][3], ve[8][3], fe[8][3];
        for (int i = 0; i < 8; ++i) {
            int32_t n = elem2node[8 * e + i];
            for (int a = 0; a < 3; ++a) {
                xe[i][a] = x[3 * n + a];
                ve[i][a] = v[3 * n + a];
            }
        }
        oracle_hex_element(xe, ve, sig + 3 * e, kappa, fe, vol + e);
        for (int i = 0; i < 8; ++i) {
            int32_t n = elem2node[8 * e + i];
            for (int a = 0; a < 3; ++a)
                f[3 * n + a] += fe[i][a];
        }
    }
}

/* -------------------------------------------------------------- adjoint */

/* Reverse sweep of euler_flux: given Fb = d(L)/d(F), accumulate
 * d(L)/d(q) into qb and d(L)/d(n) into nb.  Derived by hand from
 *   K = |rho u|^2/(2 rho), p = (gam-1)(E - K), W = rho u . n, V = W / rho. */
static void euler_flux_rev(const double *q, double nx, double ny, double gam, const double *Fb,
                           double *qb, double *nb)
{
    double rho = q[0], ru = q[1], rv = q[2], E = q[3];
    double K = 0.5 * (ru * ru + rv * rv) / rho;
    double p = (gam - 1.0) * (E - K);
    double W = ru * nx + rv * ny;
    double V = W / rho;
    /* F0 = rho V, F1 = ru V + p nx, F2 = rv V + p ny, F3 = (E + p) V */
    double Vb = Fb[0] * rho + Fb[1] * ru + Fb[2] * rv + Fb[3] * (E + p);
    double pb = Fb[1] * nx + Fb[2] * ny + Fb[3] * V;
    double rhob = Fb[0] * V;
    double rub = Fb[1] * V;
    double rvb = Fb[2] * V;
    double Eb = Fb[3] * V;
    nb[0] += Fb[1] * p;
    nb[1] += Fb[2] * p;
    /* V = W / rho */
    double Wb = Vb / rho;
    rhob -= Vb * V / rho;
    rub += Wb * nx;
    rvb += Wb * ny;
    nb[0] += Wb * ru;
    nb[1] += Wb * rv;
    /* p = (gam-1)(E - K) */
    Eb += (gam - 1.0) * pb;
    double Kb = -(gam - 1.0) * pb;
    /* K = (ru^2 + rv^2) / (2 rho) */
    rub += Kb * ru / rho;
    rvb += Kb * rv / rho;
    rhob -= Kb * K / rho;
    qb[0] += rhob;
    qb[1] += rub;
    qb[2] += rvb;
    qb[3] += Eb;
}

/* Adjoint of res_calc with x, q, adt held fixed inputs and adt not
 * differentiated:  q_bar += (d res / d q)^T res_bar,
 * x_bar += (d res / d x)^T res_bar, summed edge by edge.                  */
void oracle_res_calc_adjoint(int64_t nedge, const int32_t *edge2node, const int32_t *edge2cell,
                             const double *x, const double *q, const double *adt,
                             const double *res_bar, double *q_bar, double *x_bar, double gam,
                             double eps)
{
    for (int64_t e = 0; e < nedge; ++e) {
        int32_t a = edge2node[2 * e], b = edge2node[2 * e + 1];
        int32_t c1 = edge2cell[2 * e], c2 = edge2cell[2 * e + 1];
        double nx = x[2 * a + 1] - x[2 * b + 1];
        double ny = -(x[2 * a] - x[2 * b]);
        double mu = 0.5 * (adt[c1] + adt[c2]) * eps;
        double fb[4], hb[4];
        for (int k = 0; k < 4; ++k) {
            fb[k] = res_bar[4 * c1 + k] - res_bar[4 * c2 + k]; /* res[c1]+=f, res[c2]-=f */
            hb[k] = 0.5 * fb[k];
        }
        double nb[2] = {0.0, 0.0};
        euler_flux_rev(q + 4 * c1, nx, ny, gam, hb, q_bar + 4 * c1, nb);
        euler_flux_rev(q + 4 * c2, nx, ny, gam, hb, q_bar + 4 * c2, nb);
        for (int k = 0; k < 4; ++k) {
            q_bar[4 * c1 + k] += mu * fb[k];
            q_bar[4 * c2 + k] -= mu * fb[k];
        }
        /* nx = y_a - y_b, ny = -(x_a - x_b) */
        x_bar[2 * a + 1] += nb[0];
        x_bar[2 * b + 1] -= nb[0];
        x_bar[2 * a] -= nb[1];
        x_bar[2 * b] += nb[1];
    }
}

/* Complex-step forward res_calc: res(x + i h dx, q + i h dq) for a real step
 * h.  The flux is rational in (q, x) (no abs, no sqrt), so Im(res)/h is the
 * Jacobian-vector product J.(dq, dx) to machine precision
 * (Squire and Trapp, SIAM Review 40, 1998).  Outputs res_re, res_im are
 * [cell][4] and are overwritten.                                         */
static void euler_flux_c(const double complex *q, double complex nx, double complex ny, double gam,
                         double complex *F)
{
    double complex rho = q[0], ru = q[1], rv = q[2], E = q[3];
    double complex p = (gam - 1.0) * (E - 0.5 * (ru * ru + rv * rv) / rho);
    double complex V = (ru * nx + rv * ny) / rho;
    F[0] = rho * V;
    F[1] = ru * V + p * nx;
    F[2] = rv * V + p * ny;
    F[3] = (E + p) * V;
}

void oracle_res_calc_cstep(int64_t ncell, int64_t nedge, const int32_t *edge2node,
                           const int32_t *edge2cell, const double *x, const double *dx,
                           const double *q, const double *dq, const double *adt, double h,
                           double *res_re, double *res_im, double gam, double eps)
{
    for (int64_t i = 0; i < 4 * ncell; ++i) {
        res_re[i] = 0.0;
        res_im[i] = 0.0;
    }
    for (int64_t e = 0; e < nedge; ++e) {
        int32_t a = edge2node[2 * e], b = edge2node[2 * e + 1];
        int32_t c1 = edge2cell[2 * e], c2 = edge2cell[2 * e + 1];
        double complex xa0 = x[2 * a] + I * h * dx[2 * a], xa1 = x[2 * a + 1] + I * h * dx[2 * a + 1];
        double complex xb0 = x[2 * b] + I * h * dx[2 * b], xb1 = x[2 * b + 1] + I * h * dx[2 * b + 1];
        double complex nx = xa1 - xb1, ny = -(xa0 - xb0);
        double complex q1[4], q2[4], F1[4], F2[4];
        for (int k = 0; k < 4; ++k) {
            q1[k] = q[4 * c1 + k] + I * h * dq[4 * c1 + k];
            q2[k] = q[4 * c2 + k] + I * h * dq[4 * c2 + k];
        }
        euler_flux_c(q1, nx, ny, gam, F1);
        euler_flux_c(q2, nx, ny, gam, F2);
        double mu = 0.5 * (adt[c1] + adt[c2]) * eps;
        for (int k = 0; k < 4; ++k) {
            double complex f = 0.5 * (F1[k] + F2[k]) + mu * (q1[k] - q2[k]);
            res_re[4 * c1 + k] += creal(f);
            res_im[4 * c1 + k] += cimag(f);
            res_re[4 * c2 + k] -= creal(f);
            res_im[4 * c2 + k] -= cimag(f);
        }
    }
}

/* ------------------------------------------------------ increment-only loops */

/* Volna-style edge loop (Sec. 3.1.2).  Per edge e with cells (c1, c2),
 * direct data d = (F0, F1, F2, P, L, nx, ny) and flag:
 *   w = L (F0, F1 + P nx, F2 + P ny, P)
 *   res[c1] -= inv_area[c1] w;   res[c2] += inv_area[c2] w   unless flag
 * (a boundary edge lists its one cell twice and has flag 1). */
void oracle_space_disc(int64_t nedge, const int32_t *edge2cell, const double *edata, const int32_t *eflag,
                       const double *inv_area, double *res)
{
    for (int64_t e = 0; e < nedge; ++e) {
        const double *d = edata + 7 * e;
        const double L = d[4];
        const double w[4] = {L * d[0], L * (d[1] + d[3] * d[5]), L * (d[2] + d[3] * d[6]), L * d[3]};
        const int32_t c1 = edge2cell[2 * e], c2 = edge2cell[2 * e + 1];
        for (int k = 0; k < 4; ++k) res[4 * c1 + k] -= inv_area[c1] * w[k];
        if (!eflag[e])
            for (int k = 0; k < 4; ++k) res[4 * c2 + k] += inv_area[c2] * w[k];
    }
}

/* BookLeaf-style cell loop (Sec. 3.1.3).  Per cell c with nodes n0..n3 and
 * direct data (rho, m[4], w[4], fx[4], fy[4]):
 *   nd[n_k] += (m_k, rho w_k, fx_k, fy_k),  k = 0..3 */
void oracle_getacc(int64_t ncell, const int32_t *cell2node, const double *cdata, double *nd)
{
    for (int64_t c = 0; c < ncell; ++c) {
        const double *d = cdata + 17 * c;
        for (int k = 0; k < 4; ++k) {
            double *o = nd + 4 * (int64_t)cell2node[4 * c + k];
            o[0] += d[1 + k];
            o[1] += d[0] * d[5 + k];
            o[2] += d[9 + k];
            o[3] += d[13 + k];
        }
    }
}

/* ---------------------------------------------------------------- face flux */

/* Primitives (rho, u, v, w, p) of Q = (rho, rho u, rho v, rho w, E). */
static void aero_prim(const double *Q, double gam, double *V)
{
    V[0] = Q[0];
    V[1] = Q[1] / Q[0];
    V[2] = Q[2] / Q[0];
    V[3] = Q[3] / Q[0];
    V[4] = (gam - 1.0) * (Q[4] - 0.5 * Q[0] * (V[1] * V[1] + V[2] * V[2] + V[3] * V[3]));
}

/* Conserved state, normal Euler flux, normal velocity and sound speed of the
 * primitive state V through the unit normal n. */
static void aero_flux(const double *V, const double *n, double gam, double *Qs, double *F, double *un, double *c)
{
    const double rho = V[0], p = V[4];
    const double E = p / (gam - 1.0) + 0.5 * rho * (V[1] * V[1] + V[2] * V[2] + V[3] * V[3]);
    *un = V[1] * n[0] + V[2] * n[1] + V[3] * n[2];
    *c = sqrt(gam * p / rho);
    Qs[0] = rho;
    Qs[1] = rho * V[1];
    Qs[2] = rho * V[2];
    Qs[3] = rho * V[3];
    Qs[4] = E;
    F[0] = rho * *un;
    F[1] = rho * V[1] * *un + p * n[0];
    F[2] = rho * V[2] * *un + p * n[1];
    F[3] = rho * V[3] * *un + p * n[2];
    F[4] = (E + p) * *un;
}

/* miniAero-style face flux (Sec. 3.1.5 gives the access pattern; the
 * arithmetic is this reading).  Face f between cells c1 = face2cell[2f]
 * and c2 = face2cell[2f+1], face data (A[3], xf[3], nhat[3], dx[3]): A the
 * area normal from c1 into c2, xf the face centre, nhat = A/|A|, dx the
 * centroid of c2 minus that of c1.  Cell data (28): Q[5], gradients of the
 * primitives G[v][d] at 5 + 3 v + d, limiters phi[v] at 20 + v, centroid
 * xc at 25.
 *  1. each side: V_face = V_cell + phi (G (xf - xc)) per primitive;
 *  2. Rusanov: F_inv = |A| ((F(V_1) + F(V_2))/2 - lambda (Q(V_2) - Q(V_1))/2),
 *     lambda = max over the sides of |u.nhat| + c;
 *  3. face gradients of u, v, w and T = p/rho: the mean of the two cell
 *     gradients corrected along dx, g = g_mean + ((phi_2 - phi_1) - g_mean.dx)
 *     dx / |dx|^2 with the cell-centre values (grad T = (grad p - T grad rho)
 *     / rho per cell);
 *  4. viscous flux: tau = mu (grad u + grad u^T) - 2/3 mu (div u) I,
 *     F_v = (0, tau A, u_f . (tau A) + k grad T . A), u_f the mean of the cell
 *     velocities, k = mu gam / ((gam - 1) pr);
 *  5. F = F_inv - F_v;  res[c1] += F, res[c2] -= F  (res [cell][5]). */
void oracle_face_flux(int64_t nface, const int32_t *face2cell, const double *fdata, const double *cdata, double gam,
                      double mu, double pr, double *res)
{
    for (int64_t f = 0; f < nface; ++f) {
        const double *fd = fdata + 12 * f;
        const double *A = fd, *xf = fd + 3, *n = fd + 6, *dx = fd + 9;
        const int32_t c[2] = {face2cell[2 * f], face2cell[2 * f + 1]};
        const double area = sqrt(A[0] * A[0] + A[1] * A[1] + A[2] * A[2]);
        double Vc[2][5], Qs[2][5], F[2][5], un[2], cs[2];
        for (int s = 0; s < 2; ++s) {
            const double *cd = cdata + 28 * (int64_t)c[s];
            aero_prim(cd, gam, Vc[s]);
            const double r[3] = {xf[0] - cd[25], xf[1] - cd[26], xf[2] - cd[27]};
            double Vf[5];
            for (int v = 0; v < 5; ++v) {
                const double *g = cd + 5 + 3 * v;
                Vf[v] = Vc[s][v] + cd[20 + v] * (g[0] * r[0] + g[1] * r[1] + g[2] * r[2]);
            }
            aero_flux(Vf, n, gam, Qs[s], F[s], &un[s], &cs[s]);
        }
        const double l0 = fabs(un[0]) + cs[0], l1 = fabs(un[1]) + cs[1];
        const double lam = l0 > l1 ? l0 : l1;
        double Ft[5];
        for (int k = 0; k < 5; ++k) Ft[k] = area * (0.5 * (F[0][k] + F[1][k]) - 0.5 * lam * (Qs[1][k] - Qs[0][k]));

        /* face gradients of u, v, w (primitives 1..3) and T */
        const double *cd1 = cdata + 28 * (int64_t)c[0], *cd2 = cdata + 28 * (int64_t)c[1];
        const double dd = dx[0] * dx[0] + dx[1] * dx[1] + dx[2] * dx[2];
        double gu[3][3], gT[3];
        for (int a = 0; a < 3; ++a) {
            const double *g1 = cd1 + 5 + 3 * (1 + a), *g2 = cd2 + 5 + 3 * (1 + a);
            double gm[3];
            for (int d = 0; d < 3; ++d) gm[d] = 0.5 * (g1[d] + g2[d]);
            const double corr = ((Vc[1][1 + a] - Vc[0][1 + a]) - (gm[0] * dx[0] + gm[1] * dx[1] + gm[2] * dx[2])) / dd;
            for (int d = 0; d < 3; ++d) gu[a][d] = gm[d] + corr * dx[d];
        }
        {
            double T[2], gTc[2][3];
            const double *cds[2] = {cd1, cd2};
            for (int s = 0; s < 2; ++s) {
                T[s] = Vc[s][4] / Vc[s][0];
                for (int d = 0; d < 3; ++d) gTc[s][d] = (cds[s][5 + 12 + d] - T[s] * cds[s][5 + d]) / Vc[s][0];
            }
            double gm[3];
            for (int d = 0; d < 3; ++d) gm[d] = 0.5 * (gTc[0][d] + gTc[1][d]);
            const double corr = ((T[1] - T[0]) - (gm[0] * dx[0] + gm[1] * dx[1] + gm[2] * dx[2])) / dd;
            for (int d = 0; d < 3; ++d) gT[d] = gm[d] + corr * dx[d];
        }
        const double div = gu[0][0] + gu[1][1] + gu[2][2];
        double tA[3];
        for (int a = 0; a < 3; ++a) {
            tA[a] = 0.0;
            for (int b = 0; b < 3; ++b) {
                const double tau = mu * (gu[a][b] + gu[b][a]) - (a == b ? 2.0 / 3.0 * mu * div : 0.0);
                tA[a] += tau * A[b];
            }
        }
        const double kappa = mu * gam / ((gam - 1.0) * pr);
        double uf[3];
        for (int a = 0; a < 3; ++a) uf[a] = 0.5 * (Vc[0][1 + a] + Vc[1][1 + a]);
        const double Fv[5] = {0.0, tA[0], tA[1], tA[2],
                              uf[0] * tA[0] + uf[1] * tA[1] + uf[2] * tA[2] +
                                  kappa * (gT[0] * A[0] + gT[1] * A[1] + gT[2] * A[2])};
        for (int k = 0; k < 5; ++k) {
            res[5 * (int64_t)c[0] + k] += Ft[k] - Fv[k];
            res[5 * (int64_t)c[1] + k] -= Ft[k] - Fv[k];
        }
    }
}
