/*
 * Plain FP64 CPU oracle for the per-time-step cell/fluid update of
 * "A hyperelastic model for simulating cells in flow" (Mueller et al.).
 *
 * TEST INFRASTRUCTURE ONLY. Only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark may load this library. The CUDA path shares
 * no code, header, table or helper with it.
 *
 * Every routine is written for a reader checking it against the paper by eye:
 * no blocking, no fusion, loops in the order of the definitions, doubles
 * throughout. Layouts are the natural array-of-structures ones:
 *   vertices  x, y, u, f : [V][3]
 *   tets                 : [T][4], corner 3 is the paper's vertex 4 (origin)
 *   B                    : [T][3][3], B[k][j] = (J^-1)_kj (Sec. 3.2)
 *   corner forces        : [T][4][3]
 *   populations          : [N][19], node n = x + nx*(y + ny*z)
 *   force / velocity     : [N][3]
 *
 * Where the paper is silent (fluid operator, forcing, walls, delta kernel,
 * step order) the readings are:
 *   D3Q19, BGK with relaxation time tau, Guo forcing, halfway bounce-back with
 *   a moving-wall term (rho_0 = 1), walls half a spacing outside rows y = 0
 *   and y = ny-1, periodic x and z; trilinear two-point delta kernel, or
 *   Peskin's four-point kernel as the alternative.
 *
 * Parity pins for every function live in the non-GPU tests.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* Small 3x3 helpers                                                          */
/* ------------------------------------------------------------------------ */

static double det3(const double M[3][3]) {
    return M[0][0] * (M[1][1] * M[2][2] - M[1][2] * M[2][1])
         - M[0][1] * (M[1][0] * M[2][2] - M[1][2] * M[2][0])
         + M[0][2] * (M[1][0] * M[2][1] - M[1][1] * M[2][0]);
}

/* inverse by cofactors; caller guarantees det != 0 */
static void inv3(const double M[3][3], double R[3][3]) {
    double d = det3(M);
    R[0][0] = (M[1][1] * M[2][2] - M[1][2] * M[2][1]) / d;
    R[0][1] = (M[0][2] * M[2][1] - M[0][1] * M[2][2]) / d;
    R[0][2] = (M[0][1] * M[1][2] - M[0][2] * M[1][1]) / d;
    R[1][0] = (M[1][2] * M[2][0] - M[1][0] * M[2][2]) / d;
    R[1][1] = (M[0][0] * M[2][2] - M[0][2] * M[2][0]) / d;
    R[1][2] = (M[0][2] * M[1][0] - M[0][0] * M[1][2]) / d;
    R[2][0] = (M[1][0] * M[2][1] - M[1][1] * M[2][0]) / d;
    R[2][1] = (M[0][1] * M[2][0] - M[0][0] * M[2][1]) / d;
    R[2][2] = (M[0][0] * M[1][1] - M[0][1] * M[1][0]) / d;
}

/* ------------------------------------------------------------------------ */
/* Sec. 2: invariants, Mooney-Rivlin energy density and the derivative table  */
/* of Sec. 3.2 for one deformation gradient F (row-major F[i][j]).            */
/*                                                                            */
/* out[ 0..13] = J, T_C, T_C2, I, K, U,                                       */
/*               dU/dI, dI/dT_C, dU/dK, dK/dT_C, dI/dJ, dK/dJ, dU/dJ, dK/dT_C2 */
/* dTC[9], dJ[9], dTC2[9] = dT_C/dF_il, dJ/dF_il, dT_C2/dF_il                 */
/* P[9] = dU/dF_kl assembled by the chain rule of the force equation (Sec 3.1) */
/* ------------------------------------------------------------------------ */
void ora_mr_eval(const double *Fp, double mu1, double mu2, double kappa,
                 double *out, double *dTC, double *dJ, double *dTC2, double *P) {
    double F[3][3], C[3][3], Finv[3][3];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) F[i][j] = Fp[3 * i + j];

    /* right Cauchy-Green tensor C = F^T F */
    for (int k = 0; k < 3; ++k)
        for (int l = 0; l < 3; ++l) {
            double s = 0.0;
            for (int i = 0; i < 3; ++i) s += F[i][k] * F[i][l];
            C[k][l] = s;
        }
    double TC = C[0][0] + C[1][1] + C[2][2];
    double TC2 = 0.0; /* trace of C^2 */
    for (int k = 0; k < 3; ++k)
        for (int l = 0; l < 3; ++l) TC2 += C[k][l] * C[l][k];

    double J = det3(F);                                  /* J = det F       */
    double I = TC * pow(J, -2.0 / 3.0);                  /* I = T_C J^-2/3  */
    double K = 0.5 * (TC * TC - TC2) * pow(J, -4.0 / 3.0); /* K              */
    double U = 0.5 * mu1 * (I - 3.0) + 0.5 * mu2 * (K - 3.0) + 0.5 * kappa * (J - 1.0) * (J - 1.0);

    /* the table of Sec. 3.2, entry by entry */
    double dU_dI = 0.5 * mu1;
    double dI_dTC = pow(J, -2.0 / 3.0);
    double dU_dK = 0.5 * mu2;
    double dK_dTC = TC * pow(J, -4.0 / 3.0);
    double dI_dJ = -2.0 / 3.0 * TC * pow(J, -5.0 / 3.0);
    double dK_dJ = -2.0 / 3.0 * (TC * TC - TC2) * pow(J, -7.0 / 3.0);
    double dU_dJ = kappa * (J - 1.0);
    double dK_dTC2 = -0.5 * pow(J, -4.0 / 3.0);

    inv3(F, Finv);
    for (int i = 0; i < 3; ++i)
        for (int l = 0; l < 3; ++l) {
            dTC[3 * i + l] = 2.0 * F[i][l];
            dJ[3 * i + l] = J * Finv[l][i];
            double s = 0.0;
            for (int k = 0; k < 3; ++k) s += F[i][k] * C[k][l];
            dTC2[3 * i + l] = 4.0 * s;
        }

    /* bracket of the force equation: dU/dF_kl */
    double cTC = dU_dI * dI_dTC + dU_dK * dK_dTC;
    double cJ = dU_dI * dI_dJ + dU_dK * dK_dJ + dU_dJ;
    double cTC2 = dU_dK * dK_dTC2;
    for (int a = 0; a < 9; ++a) P[a] = cTC * dTC[a] + cJ * dJ[a] + cTC2 * dTC2[a];

    double o[14] = {J, TC, TC2, I, K, U, dU_dI, dI_dTC, dU_dK, dK_dTC, dI_dJ, dK_dJ, dU_dJ, dK_dTC2};
    memcpy(out, o, sizeof(o));
}

/* ------------------------------------------------------------------------ */
/* Sec. 3.2: per-tet Jacobian J_ik = x_i^k - x_i^4, B = J^-1, V_0, computed   */
/* once. Reading: V_0 = |det J| / 6, and a tet with det J < 0 has corners 1   */
/* and 2 swapped in place so that every stored tet is positively oriented.    */
/* Returns 0, or 1 (vertex index out of range), 2 (repeated vertex),          */
/* 3 (|det J| <= 1e-12 * (longest edge)^3). *bad_tet gets the first failing   */
/* tet.                                                                       */
/* ------------------------------------------------------------------------ */
int ora_mesh_prepare(int32_t nv, const double *x, int32_t nt, int32_t *tets,
                     double *B, double *V0, int32_t *bad_tet) {
    for (int32_t t = 0; t < nt; ++t) {
        int32_t *a = tets + 4 * t;
        for (int c = 0; c < 4; ++c)
            if (a[c] < 0 || a[c] >= nv) { *bad_tet = t; return 1; }
        for (int c = 0; c < 4; ++c)
            for (int d = c + 1; d < 4; ++d)
                if (a[c] == a[d]) { *bad_tet = t; return 2; }
        double Jm[3][3];
        for (int i = 0; i < 3; ++i)
            for (int k = 0; k < 3; ++k) Jm[i][k] = x[3 * a[k] + i] - x[3 * a[3] + i];
        double d = det3(Jm);
        double lmax = 0.0;
        for (int c = 0; c < 4; ++c)
            for (int e = c + 1; e < 4; ++e) {
                double s = 0.0;
                for (int i = 0; i < 3; ++i) {
                    double q = x[3 * a[c] + i] - x[3 * a[e] + i];
                    s += q * q;
                }
                if (s > lmax) lmax = s;
            }
        lmax = sqrt(lmax);
        if (fabs(d) <= 1e-12 * lmax * lmax * lmax) { *bad_tet = t; return 3; }
        if (d < 0.0) {
            int32_t tmp = a[0]; a[0] = a[1]; a[1] = tmp;
            for (int i = 0; i < 3; ++i) {
                double q = Jm[i][0]; Jm[i][0] = Jm[i][1]; Jm[i][1] = q;
            }
            d = -d;
        }
        double Bi[3][3];
        inv3(Jm, Bi);
        for (int k = 0; k < 3; ++k)
            for (int j = 0; j < 3; ++j) B[9 * t + 3 * k + j] = Bi[k][j];
        V0[t] = d / 6.0;
    }
    *bad_tet = -1;
    return 0;
}

/* Vertex -> (tet, corner) incidence in compressed rows; entries 4*t + c in  */
/* ascending order within each row (the order of the vertex force sum).       */
void ora_csr(int32_t nv, int32_t nt, const int32_t *tets, int32_t *ptr, int32_t *idx) {
    for (int32_t v = 0; v <= nv; ++v) ptr[v] = 0;
    for (int32_t t = 0; t < nt; ++t)
        for (int c = 0; c < 4; ++c) ptr[tets[4 * t + c] + 1] += 1;
    for (int32_t v = 0; v < nv; ++v) ptr[v + 1] += ptr[v];
    int32_t *fill = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nv > 0 ? nv : 1));
    for (int32_t v = 0; v < nv; ++v) fill[v] = ptr[v];
    for (int32_t t = 0; t < nt; ++t)
        for (int c = 0; c < 4; ++c) idx[fill[tets[4 * t + c]]++] = 4 * t + c;
    free(fill);
}

/* ------------------------------------------------------------------------ */
/* Sec. 3.1-3.2: nodal elastic force f_i^a = -V_0 dU/du_i^a of every tet.     */
/* A_ik = u_i^k - u_i^4; F = I + A B; P = dU/dF from ora_mr_eval; then        */
/* dF_kl/du_i^a = delta_ki B_ml (delta_ma - delta_4a), summed over k, l, m.   */
/* Material per tet through cell[t]: mu_1 = w mu, mu_2 = (1-w) mu (Sec. 2).   */
/* Writes corner forces fc [T][4][3] and, if energy != NULL, V_0 U per tet.   */
/* Tets in [t0, t1) only.                                                     */
/* ------------------------------------------------------------------------ */
void ora_tet_force(int32_t t0, int32_t t1, const int32_t *tets, const double *B, const double *V0,
                   const double *u, const int32_t *cell, const double *mu, const double *kappa,
                   const double *w, double *fc, double *energy) {
    for (int32_t t = t0; t < t1; ++t) {
        const int32_t *a = tets + 4 * t;
        const double *Bt = B + 9 * t;
        double A[3][3];
        for (int i = 0; i < 3; ++i)
            for (int k = 0; k < 3; ++k) A[i][k] = u[3 * a[k] + i] - u[3 * a[3] + i];
        double F[9];
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
                double s = (i == j) ? 1.0 : 0.0;
                for (int k = 0; k < 3; ++k) s += A[i][k] * Bt[3 * k + j];
                F[3 * i + j] = s;
            }
        int32_t c = cell[t];
        double mu1 = w[c] * mu[c], mu2 = (1.0 - w[c]) * mu[c];
        double sc[14], dTC[9], dJ[9], dTC2[9], P[9];
        ora_mr_eval(F, mu1, mu2, kappa[c], sc, dTC, dJ, dTC2, P);
        for (int al = 0; al < 4; ++al)
            for (int i = 0; i < 3; ++i) {
                double s = 0.0;
                for (int k = 0; k < 3; ++k)
                    for (int l = 0; l < 3; ++l) {
                        if (k != i) continue; /* delta_ki */
                        for (int m = 0; m < 3; ++m) {
                            double dm = (m == al ? 1.0 : 0.0) - (al == 3 ? 1.0 : 0.0);
                            s += P[3 * k + l] * Bt[3 * m + l] * dm;
                        }
                    }
                fc[12 * t + 3 * al + i] = -V0[t] * s;
            }
        if (energy) energy[t] = V0[t] * sc[5];
    }
}

/* Vertex force: sum of the corner forces of every incident (tet, corner),   */
/* in the ascending order of the incidence rows.                              */
void ora_gather(int32_t v0, int32_t v1, const int32_t *ptr, const int32_t *idx,
                const double *fc, double *f) {
    for (int32_t v = v0; v < v1; ++v) {
        double s[3] = {0.0, 0.0, 0.0};
        for (int32_t e = ptr[v]; e < ptr[v + 1]; ++e)
            for (int i = 0; i < 3; ++i) s[i] += fc[3 * idx[e] + i];
        for (int i = 0; i < 3; ++i) f[3 * v + i] = s[i];
    }
}

/* ------------------------------------------------------------------------ */
/* Immersed boundary (Sec. 6; kernel not given in the paper): a separable    */
/* delta_h(r) = phi(r_x) phi(r_y) phi(r_z) of support width 2 or 4 nodes per  */
/* axis:                                                                      */
/*   width 2, trilinear: phi(r) = max(0, 1 - |r|);                            */
/*   width 4, Peskin's four-point kernel (Acta Numerica 2002, Sec. 6):        */
/*     phi(r) = (3 - 2|r| + sqrt(1 + 4|r| - 4 r^2)) / 8    for |r| <= 1,      */
/*              (5 - 2|r| - sqrt(-7 + 12|r| - 4 r^2)) / 8  for 1 <= |r| <= 2, */
/*              0 otherwise.                                                  */
/* The support of a point p on one axis is the nodes floor(p) - (width/2 - 1) */
/* + {0, .., width-1}; x and z wrap periodically, y must stay in [0, ny-1].   */
/* ------------------------------------------------------------------------ */
static double phi2(double r) {
    r = fabs(r);
    return r < 1.0 ? 1.0 - r : 0.0;
}

static double phi4(double r) {
    r = fabs(r);
    if (r <= 1.0) return (3.0 - 2.0 * r + sqrt(1.0 + 4.0 * r - 4.0 * r * r)) / 8.0;
    if (r <= 2.0) return (5.0 - 2.0 * r - sqrt(-7.0 + 12.0 * r - 4.0 * r * r)) / 8.0;
    return 0.0;
}

static double phi(double r, int width) { return width == 4 ? phi4(r) : phi2(r); }

static int wrap(int i, int n) {
    int m = i % n;
    return m < 0 ? m + n : m;
}

/* F(x) += sum_v f_v delta_h(x - y_v). Returns the number of vertices whose  */
/* support leaves 0 <= y <= ny-1 (those are skipped).                         */
int ora_spread(int32_t v0, int32_t v1, const double *y, const double *f,
               int nx, int ny, int nz, int width, double *Fn) {
    int bad = 0;
    for (int32_t v = v0; v < v1; ++v) {
        const double *p = y + 3 * v;
        int lo = width / 2 - 1;
        int bx = (int)floor(p[0]) - lo, by = (int)floor(p[1]) - lo, bz = (int)floor(p[2]) - lo;
        if (by < 0 || by + width - 1 > ny - 1) { ++bad; continue; }
        for (int dz = 0; dz < width; ++dz)
            for (int dy = 0; dy < width; ++dy)
                for (int dx = 0; dx < width; ++dx) {
                    int X = bx + dx, Y = by + dy, Z = bz + dz;
                    double d = phi(X - p[0], width) * phi(Y - p[1], width) * phi(Z - p[2], width);
                    size_t n = (size_t)wrap(X, nx) + (size_t)nx * ((size_t)Y + (size_t)ny * (size_t)wrap(Z, nz));
                    for (int i = 0; i < 3; ++i) Fn[3 * n + i] += d * f[3 * v + i];
                }
    }
    return bad;
}

/* v(y_v) = sum_x u(x) delta_h(x - y_v). Same support rule as ora_spread.    */
int ora_interp(int32_t v0, int32_t v1, const double *y, const double *un,
               int nx, int ny, int nz, int width, double *vel) {
    int bad = 0;
    for (int32_t v = v0; v < v1; ++v) {
        const double *p = y + 3 * v;
        int lo = width / 2 - 1;
        int bx = (int)floor(p[0]) - lo, by = (int)floor(p[1]) - lo, bz = (int)floor(p[2]) - lo;
        double s[3] = {0.0, 0.0, 0.0};
        if (by < 0 || by + width - 1 > ny - 1) {
            ++bad;
        } else {
            for (int dz = 0; dz < width; ++dz)
                for (int dy = 0; dy < width; ++dy)
                    for (int dx = 0; dx < width; ++dx) {
                        int X = bx + dx, Y = by + dy, Z = bz + dz;
                        double d = phi(X - p[0], width) * phi(Y - p[1], width) * phi(Z - p[2], width);
                        size_t n = (size_t)wrap(X, nx) + (size_t)nx * ((size_t)Y + (size_t)ny * (size_t)wrap(Z, nz));
                        for (int i = 0; i < 3; ++i) s[i] += d * un[3 * n + i];
                    }
        }
        for (int i = 0; i < 3; ++i) vel[3 * v + i] = s[i];
    }
    return bad;
}

/* ------------------------------------------------------------------------ */
/* Lattice Boltzmann fluid (Sec. 6 uses ESPResSo's LB; the operator is not    */
/* stated). D3Q19 with c_s^2 = 1/3; order: rest, +x, -x, +y, -y, +z, -z, then */
/* the 12 vectors with two nonzero components in lexicographic order.         */
/* ------------------------------------------------------------------------ */
static const int CV[19][3] = {
    {0, 0, 0},
    {1, 0, 0}, {-1, 0, 0}, {0, 1, 0}, {0, -1, 0}, {0, 0, 1}, {0, 0, -1},
    {-1, -1, 0}, {-1, 0, -1}, {-1, 0, 1}, {-1, 1, 0}, {0, -1, -1}, {0, -1, 1},
    {0, 1, -1}, {0, 1, 1}, {1, -1, 0}, {1, 0, -1}, {1, 0, 1}, {1, 1, 0}};

static double weight(int i) {
    int s = abs(CV[i][0]) + abs(CV[i][1]) + abs(CV[i][2]);
    return s == 0 ? 1.0 / 3.0 : (s == 1 ? 1.0 / 18.0 : 1.0 / 36.0);
}

static int opposite(int i) {
    for (int j = 0; j < 19; ++j)
        if (CV[j][0] == -CV[i][0] && CV[j][1] == -CV[i][1] && CV[j][2] == -CV[i][2]) return j;
    return -1;
}

void ora_lbm_velocities(int32_t *c, double *w) {
    for (int i = 0; i < 19; ++i) {
        for (int a = 0; a < 3; ++a) c[3 * i + a] = CV[i][a];
        w[i] = weight(i);
    }
}

/* f^eq_i = w_i rho [1 + 3 c.u + 9/2 (c.u)^2 - 3/2 u.u] */
static double feq(int i, double rho, const double u[3]) {
    double cu = CV[i][0] * u[0] + CV[i][1] * u[1] + CV[i][2] * u[2];
    double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    return weight(i) * rho * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * uu);
}

/* Equilibrium at rho, u on every node (initial state). */
void ora_lbm_equilibrium(int64_t n_nodes, double rho, const double *u, double *f) {
    for (int64_t n = 0; n < n_nodes; ++n)
        for (int i = 0; i < 19; ++i) f[19 * n + i] = feq(i, rho, u);
}

/* One pull stream + collide for nodes [n0, n1). fin holds the post-collision */
/* populations of the previous step; fout gets the new post-collision ones.   */
/*  stream: f_i(x) = fin_i(x - c_i); x - c_i beyond a wall is bounced back:   */
/*          f_i(x) = fin_ibar(x) + 6 w_i rho_0 (c_i . u_wall), rho_0 = 1.     */
/*  moments: rho = sum f_i; rho u = sum c_i f_i + F/2 (F = Fn(x) + g).        */
/*  collide (BGK + Guo): f*_i = f_i - (f_i - f^eq_i)/tau                      */
/*          + (1 - 1/(2 tau)) w_i [3 (c_i - u) + 9 (c_i . u) c_i] . F.        */
/* rho_out / u_out (if non-NULL) receive rho and u of the collision.          */
void ora_lbm_step(int nx, int ny, int nz, double tau, double uw_lo, double uw_hi,
                  const double *g, const double *fin, const double *Fn, double *fout,
                  double *rho_out, double *u_out, int64_t n0, int64_t n1) {
    for (int64_t n = n0; n < n1; ++n) {
        int x = (int)(n % nx), y = (int)((n / nx) % ny), z = (int)(n / ((int64_t)nx * ny));
        double f[19];
        for (int i = 0; i < 19; ++i) {
            int sx = x - CV[i][0], sy = y - CV[i][1], sz = z - CV[i][2];
            if (sy < 0 || sy > ny - 1) {
                double uw = sy < 0 ? uw_lo : uw_hi; /* wall moves along x */
                f[i] = fin[19 * n + opposite(i)] + 6.0 * weight(i) * 1.0 * (CV[i][0] * uw);
            } else {
                int64_t s = (int64_t)wrap(sx, nx) + (int64_t)nx * (sy + (int64_t)ny * wrap(sz, nz));
                f[i] = fin[19 * s + i];
            }
        }
        double Fx[3] = {0.0, 0.0, 0.0};
        for (int a = 0; a < 3; ++a) {
            if (Fn) Fx[a] += Fn[3 * n + a];
            if (g) Fx[a] += g[a];
        }
        double rho = 0.0, mom[3] = {0.0, 0.0, 0.0};
        for (int i = 0; i < 19; ++i) {
            rho += f[i];
            for (int a = 0; a < 3; ++a) mom[a] += CV[i][a] * f[i];
        }
        double u[3];
        for (int a = 0; a < 3; ++a) u[a] = (mom[a] + 0.5 * Fx[a]) / rho;
        for (int i = 0; i < 19; ++i) {
            double cu = CV[i][0] * u[0] + CV[i][1] * u[1] + CV[i][2] * u[2];
            double src = 0.0;
            for (int a = 0; a < 3; ++a) src += (3.0 * (CV[i][a] - u[a]) + 9.0 * cu * CV[i][a]) * Fx[a];
            src *= (1.0 - 0.5 / tau) * weight(i);
            fout[19 * n + i] = f[i] - (f[i] - feq(i, rho, u)) / tau + src;
        }
        if (rho_out) rho_out[n] = rho;
        if (u_out)
            for (int a = 0; a < 3; ++a) u_out[3 * n + a] = u[a];
    }
}
