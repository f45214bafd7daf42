/*
 * femoracle.c -- plain, slow, obviously-correct FP64 CPU oracle of the discrete
 * energy J(v) = J_grad(v) - b.v and its gradients over P1 triangles / tetrahedra
 * (Moskovka & Valdman, "Fast MATLAB evaluation of nonlinear energies using FEM in 2D
 * and 3D: Nodal elements", arXiv 2109.01158).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the reference against which the CUDA path is
 * checked.  Only the test-suite, the smoke check and the benchmark's CPU-baseline leg
 * may load it.  It shares no code, header, table or helper with the CUDA library.
 *
 * Conventions (all 0-based):
 *   coords[i*dim + m]          node i, coordinate m                  (nodes2coord)
 *   elems[e*(dim+1) + l]       global node of local node l of elem e  (elems2nodes, I_LG)
 *   dphi[(e*(dim+1) + l)*dim+m] d(phi_{e,l})/d(x_m) on element e       (dphi)
 *   vol[e]                     |T_e|                                   (volumes)
 *   v[i*d + j], b[i*d + j]     interleaved dof order n = d*i + j       (eq. bvvectors)
 *   dirichlet[i*d + j]         1 = fixed dof (dofsDirichlet), 0 = free (dofsMinim)
 *
 * Readings of the paper taken here (each explained where it is used):
 *   - J = J_grad - b.v and grad J = grad J_grad - b, b^(j) = M f^(j)   (problem
 *     statements Sec. 1; Sec. 3.2 eq. linearTerm2 written with a + sign is read as the
 *     inner product that is subtracted).
 *   - Neo-Hookean: v is the deformation, F = grad v; F is formed as
 *     F = I + sum_l (v_l - X_l) grad(phi_l)^T, which equals eq. (Dv) exactly in real
 *     arithmetic because sum_l X_l grad(phi_l)^T = I for P1 elements.
 *   - det F <= 0: W = +Inf and the status OR_EDOMAIN (the paper's log would be complex).
 *   - p-Laplacian: W = (1/p) |grad v|^p; its derivative is |grad v|^(p-2) grad v, set to
 *     0 where grad v = 0.  Model OR_PLAPLACE_LP reads |grad v|^p with the l^p norm of the
 *     gradient, W = (1/p) sum_m |dv/dx_m|^p, the reading under which the minima printed in
 *     the table of Benchmark 6 are reproduced.
 *   - The gradient is returned for every dof, with Dirichlet dofs set to 0 (Remark 1
 *     restricts it to the free dofs; the restriction is g[free]).
 *   - Patch sums are plain sums over the patch in increasing element order (the
 *     cumulative-sum/difference trick of Sec. 6.1 is not used: its rounding grows with
 *     the running total).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_OK 0
#define OR_EINVAL 1
#define OR_ENOMEM 2
#define OR_EDOMAIN 4

#define OR_PLAPLACE 0
#define OR_NEOHOOKE 1
#define OR_PLAPLACE_LP 2   /* W = (1/p) sum_m |dv/dx_m|^p: |grad v|^p read with the l^p norm */

/* ------------------------------------------------------------------------------ */
/* Neumaier's compensated summation (Neumaier 1974), used for the two global sums.  */
/* ------------------------------------------------------------------------------ */
typedef struct { double s, c; } or_sum;

static void or_sum_add(or_sum* a, double x) {
    double t = a->s + x;
    if (fabs(a->s) >= fabs(x)) a->c += (a->s - t) + x;
    else a->c += (x - t) + a->s;
    a->s = t;
}
static double or_sum_get(const or_sum* a) { return a->s + a->c; }

/* ------------------------------------------------------------------------------ */
/* Mesh precompute: volumes and P1 shape-function gradients (Sec. 4.1).           */
/* With B = [x_1-x_0, ..., x_dim-x_0] (columns), the barycentric coordinates of x are */
/* xi = B^{-1}(x - x_0); phi_l = xi_l for l >= 1 and phi_0 = 1 - sum xi, so          */
/* grad(phi_l) is row l of B^{-1} and grad(phi_0) = -sum_l grad(phi_l).              */
/* |T| = |det B| / dim!.                                                            */
/* ------------------------------------------------------------------------------ */
int or_precompute(int dim, int64_t nn, const double* coords, int64_t ne,
                  const int32_t* elems, double* dphi, double* vol) {
    if (dim != 2 && dim != 3) return OR_EINVAL;
    int status = OR_OK;
    for (int64_t e = 0; e < ne; ++e) {
        const int32_t* en = elems + e * (dim + 1);
        for (int l = 0; l <= dim; ++l)
            if (en[l] < 0 || en[l] >= nn) return OR_EINVAL;
        double B[3][3] = {{0}}, inv[3][3] = {{0}}, det;
        const double* x0 = coords + (int64_t)en[0] * dim;
        for (int k = 1; k <= dim; ++k) {
            const double* xk = coords + (int64_t)en[k] * dim;
            for (int m = 0; m < dim; ++m) B[m][k - 1] = xk[m] - x0[m];
        }
        if (dim == 2) {
            det = B[0][0] * B[1][1] - B[0][1] * B[1][0];
            inv[0][0] = B[1][1] / det;
            inv[0][1] = -B[0][1] / det;
            inv[1][0] = -B[1][0] / det;
            inv[1][1] = B[0][0] / det;
            vol[e] = fabs(det) / 2.0;
        } else {
            /* cofactors C[a][c] = (-1)^(a+c) * minor(a,c); inverse = C^T / det */
            double C[3][3];
            for (int a = 0; a < 3; ++a)
                for (int c = 0; c < 3; ++c) {
                    int r0 = (a + 1) % 3, r1 = (a + 2) % 3;
                    int c0 = (c + 1) % 3, c1 = (c + 2) % 3;
                    /* cyclic index choice already carries the sign (-1)^(a+c) */
                    C[a][c] = B[r0][c0] * B[r1][c1] - B[r0][c1] * B[r1][c0];
                }
            det = B[0][0] * C[0][0] + B[0][1] * C[0][1] + B[0][2] * C[0][2];
            for (int a = 0; a < 3; ++a)
                for (int c = 0; c < 3; ++c) inv[a][c] = C[c][a] / det;
            vol[e] = fabs(det) / 6.0;
        }
        if (det == 0.0 || !isfinite(det)) status = OR_EINVAL;
        double* de = dphi + e * (dim + 1) * dim;
        for (int m = 0; m < dim; ++m) de[m] = 0.0;
        for (int l = 1; l <= dim; ++l)
            for (int m = 0; m < dim; ++m) {
                de[l * dim + m] = inv[l - 1][m];
                de[m] -= inv[l - 1][m];
            }
    }
    return status;
}

/* ------------------------------------------------------------------------------ */
/* Nodal patches T^i = {T : N_i in T} (Sec. 3, Sec. 4.2) as a CSR:                 */
/* row_ptr[i]..row_ptr[i+1]-1 hold the entries e*(dim+1)+l with elems[e][l] == i,    */
/* in increasing element order.  row_ptr plays the role of the offsets p_i.         */
/* ------------------------------------------------------------------------------ */
int or_build_patches(int dim, int64_t nn, int64_t ne, const int32_t* elems,
                     int64_t* row_ptr, int64_t* ent) {
    const int k = dim + 1;
    for (int64_t i = 0; i <= nn; ++i) row_ptr[i] = 0;
    for (int64_t e = 0; e < ne; ++e)
        for (int l = 0; l < k; ++l) {
            int32_t i = elems[e * k + l];
            if (i < 0 || i >= nn) return OR_EINVAL;
            row_ptr[i + 1] += 1;
        }
    for (int64_t i = 0; i < nn; ++i) row_ptr[i + 1] += row_ptr[i];
    int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (size_t)(nn > 0 ? nn : 1));
    if (!fill) return OR_ENOMEM;
    for (int64_t i = 0; i < nn; ++i) fill[i] = row_ptr[i];
    for (int64_t e = 0; e < ne; ++e)
        for (int l = 0; l < k; ++l) {
            int32_t i = elems[e * k + l];
            ent[fill[i]++] = e * k + l;
        }
    free(fill);
    return OR_OK;
}

/* ------------------------------------------------------------------------------ */
/* Linear term: b^(j) = M f^(j) (eq. mass2D, linearTerm2) with the P1 element mass  */
/* matrix M^T_{ab} = |T| (1 + delta_ab) / ((dim+1)(dim+2)).                         */
/* ------------------------------------------------------------------------------ */
void or_load_vector(int dim, int d, int64_t nn, int64_t ne, const int32_t* elems,
                    const double* vol, const double* f, double* b) {
    const int k = dim + 1;
    for (int64_t n = 0; n < nn * d; ++n) b[n] = 0.0;
    if (!f) return;
    for (int64_t e = 0; e < ne; ++e) {
        const int32_t* en = elems + e * k;
        double w = vol[e] / (double)((dim + 1) * (dim + 2));
        for (int a = 0; a < k; ++a)
            for (int j = 0; j < d; ++j) {
                double s = 0.0;
                for (int c = 0; c < k; ++c)
                    s += (a == c ? 2.0 : 1.0) * f[(int64_t)en[c] * d + j];
                b[(int64_t)en[a] * d + j] += w * s;
            }
    }
}

/* ------------------------------------------------------------------------------ */
/* Element kinematics.  F is d x dim (row j = gradient of component j).           */
/* Neo-Hookean: F = I + sum_l u_l grad(phi_l)^T, u_l = v_l - X_l  (eq. Dv).         */
/* p-Laplacian: F (1 x dim) = sum_l v_l grad(phi_l)^T                (eq. Dv, d=1). */
/* ------------------------------------------------------------------------------ */
typedef struct {
    int model, dim, d;
    double p, C1, D1;
    const double* coords;
    const int32_t* elems;
    const double* dphi;
    const double* vol;
} or_mesh;

static void or_local_values(const or_mesh* M, int64_t e, const double* v, double uloc[4][3]) {
    const int k = M->dim + 1;
    const int32_t* en = M->elems + e * k;
    for (int l = 0; l < k; ++l)
        for (int j = 0; j < M->d; ++j) {
            double vv = v[(int64_t)en[l] * M->d + j];
            if (M->model == OR_NEOHOOKE) vv -= M->coords[(int64_t)en[l] * M->dim + j];
            uloc[l][j] = vv;
        }
}

static void or_element_F(const or_mesh* M, int64_t e, double uloc[4][3], double F[3][3]) {
    const int k = M->dim + 1;
    const double* de = M->dphi + e * k * M->dim;
    for (int j = 0; j < M->d; ++j)
        for (int m = 0; m < M->dim; ++m) {
            double s = 0.0;
            for (int l = 0; l < k; ++l) s += uloc[l][j] * de[l * M->dim + m];
            F[j][m] = (M->model == OR_NEOHOOKE && j == m) ? 1.0 + s : s;
        }
}

/* determinant of F (Sarrus' rule in 3D, as in the density listing of Sec. 5) */
static double or_det(int dim, double F[3][3]) {
    if (dim == 2) return F[0][0] * F[1][1] - F[0][1] * F[1][0];
    return F[0][0] * F[1][1] * F[2][2] + F[0][2] * F[1][0] * F[2][1]
         + F[0][1] * F[1][2] * F[2][0] - F[0][2] * F[1][1] * F[2][0]
         - F[0][1] * F[1][0] * F[2][2] - F[0][0] * F[1][2] * F[2][1];
}

/* density W(F): eq. (neoHook) or the p-Laplacian integrand of eq. (pLaplacian) */
static double or_density(const or_mesh* M, double F[3][3], int* dom_err) {
    if (M->model == OR_NEOHOOKE) {
        double I1 = 0.0;
        for (int j = 0; j < M->dim; ++j)
            for (int m = 0; m < M->dim; ++m) I1 += F[j][m] * F[j][m];
        double det = or_det(M->dim, F);
        if (!(det > 0.0)) { *dom_err = 1; return INFINITY; }
        return M->C1 * (I1 - (double)M->dim - 2.0 * log(det)) + M->D1 * (det - 1.0) * (det - 1.0);
    }
    if (M->model == OR_PLAPLACE_LP) {
        double s = 0.0;
        for (int m = 0; m < M->dim; ++m) s += pow(fabs(F[0][m]), M->p);
        return s / M->p;
    }
    double s = 0.0;
    for (int m = 0; m < M->dim; ++m) s += F[0][m] * F[0][m];
    return pow(s, M->p / 2.0) / M->p;
}

/* dW/dF (d x dim).  Neo-Hookean (Sec. 6.2):
 *   dW/dF_jm = C1 (dI1/dF_jm - (2/det F) ddet/dF_jm) + 2 D1 (det F - 1) ddet/dF_jm,
 *   dI1/dF_jm = 2 F_jm,  ddet/dF_jm = (-1)^(j+m) det(F^sub_jm)  (row/column expansion).
 * p-Laplacian: dW/dF_m = |F|^(p-2) F_m (0 where F = 0). */
static void or_dW(const or_mesh* M, double F[3][3], double P[3][3], int* dom_err) {
    if (M->model == OR_NEOHOOKE) {
        const int dim = M->dim;
        double det = or_det(dim, F);
        if (!(det > 0.0)) *dom_err = 1;
        for (int j = 0; j < dim; ++j)
            for (int m = 0; m < dim; ++m) {
                double minor;
                if (dim == 2) {
                    minor = F[1 - j][1 - m];
                } else {
                    int r[2], c[2], nr = 0, nc = 0;
                    for (int a = 0; a < 3; ++a) if (a != j) r[nr++] = a;
                    for (int a = 0; a < 3; ++a) if (a != m) c[nc++] = a;
                    minor = F[r[0]][c[0]] * F[r[1]][c[1]] - F[r[0]][c[1]] * F[r[1]][c[0]];
                }
                double ddet = ((j + m) % 2 == 0) ? minor : -minor;
                P[j][m] = M->C1 * (2.0 * F[j][m] - (2.0 / det) * ddet)
                        + 2.0 * M->D1 * (det - 1.0) * ddet;
            }
        return;
    }
    if (M->model == OR_PLAPLACE_LP) {   /* dW/dF_m = |F_m|^(p-2) F_m, 0 where F_m = 0 */
        for (int m = 0; m < M->dim; ++m)
            P[0][m] = (F[0][m] != 0.0) ? pow(fabs(F[0][m]), M->p - 2.0) * F[0][m] : 0.0;
        return;
    }
    double s = 0.0;
    for (int m = 0; m < M->dim; ++m) s += F[0][m] * F[0][m];
    double c = (s > 0.0) ? pow(s, (M->p - 2.0) / 2.0) : 0.0;
    for (int m = 0; m < M->dim; ++m) P[0][m] = c * F[0][m];
}

static int or_check_model(int model, int dim, int d) {
    if (dim != 2 && dim != 3) return 0;
    if (model == OR_NEOHOOKE) return d == dim;
    if (model == OR_PLAPLACE || model == OR_PLAPLACE_LP) return d == 1;
    return 0;
}

/* ------------------------------------------------------------------------------ */
/* Energy (Sec. 5): J = sum_k |T_k| W(grad v|T_k) - b.v   (eqs. Denergy, linearTerm3) */
/* ------------------------------------------------------------------------------ */
int or_energy(int model, double p, double C1, double D1, int dim, int d, int64_t nn,
              const double* coords, int64_t ne, const int32_t* elems, const double* dphi,
              const double* vol, const double* b, const double* v, double* J_out,
              double* dens) {
    if (!or_check_model(model, dim, d)) return OR_EINVAL;
    or_mesh M = {model, dim, d, p, C1, D1, coords, elems, dphi, vol};
    or_sum sg = {0, 0}, sl = {0, 0};
    int dom_err = 0;
    for (int64_t e = 0; e < ne; ++e) {
        double uloc[4][3], F[3][3];
        or_local_values(&M, e, v, uloc);
        or_element_F(&M, e, uloc, F);
        double W = or_density(&M, F, &dom_err);
        if (dens) dens[e] = W;
        or_sum_add(&sg, vol[e] * W);
    }
    if (b)
        for (int64_t n = 0; n < nn * d; ++n) or_sum_add(&sl, b[n] * v[n]);
    *J_out = dom_err ? INFINITY : or_sum_get(&sg) - or_sum_get(&sl);
    return dom_err ? OR_EDOMAIN : OR_OK;
}

/* ------------------------------------------------------------------------------ */
/* Exact gradient (Sec. 6.2): dJ_grad/dv_n = sum_{T in patch} |T| sum_{j,m}         */
/* dW/dF_jm dF_jm/dv_n, with dF_jm/dv_{(i,j')} = delta_{j j'} dphi_l/dx_m for the    */
/* local index l of node i in T (eq. dWFv).  Then g = grad J_grad - b, 0 on Dirichlet. */
/* ------------------------------------------------------------------------------ */
int or_gradient_exact(int model, double p, double C1, double D1, int dim, int d, int64_t nn,
                      const double* coords, int64_t ne, const int32_t* elems,
                      const double* dphi, const double* vol, const double* b,
                      const uint8_t* dirichlet, const int64_t* row_ptr, const int64_t* ent,
                      const double* v, double* g) {
    if (!or_check_model(model, dim, d)) return OR_EINVAL;
    or_mesh M = {model, dim, d, p, C1, D1, coords, elems, dphi, vol};
    const int k = dim + 1;
    double* r = (double*)malloc(sizeof(double) * (size_t)(ne > 0 ? ne * k * d : 1));
    if (!r) return OR_ENOMEM;
    int dom_err = 0;
    for (int64_t e = 0; e < ne; ++e) {
        double uloc[4][3], F[3][3], P[3][3];
        or_local_values(&M, e, v, uloc);
        or_element_F(&M, e, uloc, F);
        or_dW(&M, F, P, &dom_err);
        const double* de = dphi + e * k * dim;
        for (int l = 0; l < k; ++l)
            for (int j = 0; j < d; ++j) {
                double s = 0.0;
                for (int m = 0; m < dim; ++m) s += P[j][m] * de[l * dim + m];
                r[(e * k + l) * d + j] = vol[e] * s;
            }
    }
    for (int64_t i = 0; i < nn; ++i)
        for (int j = 0; j < d; ++j) {
            double s = 0.0;
            for (int64_t q = row_ptr[i]; q < row_ptr[i + 1]; ++q) s += r[ent[q] * d + j];
            int64_t n = i * d + j;
            s -= b ? b[n] : 0.0;
            g[n] = (dirichlet && dirichlet[n]) ? 0.0 : s;
        }
    free(r);
    return dom_err ? OR_EDOMAIN : OR_OK;
}

/* ------------------------------------------------------------------------------ */
/* Central-difference gradient over nodal patches (Sec. 6.1, eqs. CD, CDS, jgradpm,  */
/* sumpatch): for dof n = d*i + j,                                                 */
/*   g_n = ( sum_{T in T^i} |T| W(F_T^{+}) - sum_{T in T^i} |T| W(F_T^{-}) ) / (2 eps) - b_n */
/* where F_T^{+-} is F_T with row j recomputed from the nodal values in which the   */
/* value at node i, component j, is shifted by +-eps (the rest of F is unchanged).  */
/* dofs == NULL: every dof, written to g[n] (Dirichlet dofs 0).                    */
/* Otherwise g[q] for dof dofs[q].                                                 */
/* ------------------------------------------------------------------------------ */
int or_gradient_fd(int model, double p, double C1, double D1, int dim, int d, int64_t nn,
                   const double* coords, int64_t ne, const int32_t* elems,
                   const double* dphi, const double* vol, const double* b,
                   const uint8_t* dirichlet, const int64_t* row_ptr, const int64_t* ent,
                   const double* v, double eps, const int64_t* dofs, int64_t ndofs,
                   double* g) {
    if (!or_check_model(model, dim, d)) return OR_EINVAL;
    or_mesh M = {model, dim, d, p, C1, D1, coords, elems, dphi, vol};
    const int k = dim + 1;
    int64_t count = dofs ? ndofs : nn * d;
    int dom_err = 0;
    for (int64_t q = 0; q < count; ++q) {
        int64_t n = dofs ? dofs[q] : q;
        if (n < 0 || n >= nn * d) return OR_EINVAL;
        int64_t i = n / d;
        int j = (int)(n % d);
        if (dirichlet && dirichlet[n]) { g[q] = 0.0; continue; }
        double sp = 0.0, sm = 0.0;
        for (int64_t t = row_ptr[i]; t < row_ptr[i + 1]; ++t) {
            int64_t e = ent[t] / k;
            int lc = (int)(ent[t] % k);
            double uloc[4][3], F[3][3], Fp[3][3], Fm[3][3];
            or_local_values(&M, e, v, uloc);
            or_element_F(&M, e, uloc, F);
            const double* de = dphi + e * k * dim;
            for (int a = 0; a < 3; ++a)
                for (int c = 0; c < 3; ++c) { Fp[a][c] = F[a][c]; Fm[a][c] = F[a][c]; }
            for (int m = 0; m < dim; ++m) {
                double sP = 0.0, sM = 0.0;
                for (int l = 0; l < k; ++l) {
                    double ul = uloc[l][j];
                    sP += (l == lc ? ul + eps : ul) * de[l * dim + m];
                    sM += (l == lc ? ul - eps : ul) * de[l * dim + m];
                }
                int diag = (model == OR_NEOHOOKE && j == m);
                Fp[j][m] = diag ? 1.0 + sP : sP;
                Fm[j][m] = diag ? 1.0 + sM : sM;
            }
            sp += vol[e] * or_density(&M, Fp, &dom_err);
            sm += vol[e] * or_density(&M, Fm, &dom_err);
        }
        g[q] = (sp - sm) / (2.0 * eps) - (b ? b[n] : 0.0);
    }
    return dom_err ? OR_EDOMAIN : OR_OK;
}

/* ------------------------------------------------------------------------------ */
/* Hessian-vector product: Hw = d/dt grad J(v + t w) at t = 0 on the free dofs, i.e.  */
/* for every element the directional derivative of dW/dF along dF = sum_l w_l        */
/* grad(phi_l)^T, contracted with grad(phi_l) and gathered over the patches like the */
/* exact gradient (Sec. 6.2).  The linear term b.v has no second derivative.  Entries */
/* of w on Dirichlet dofs are taken as 0 and Dirichlet rows of Hw are 0 (the Hessian  */
/* of J restricted to the free dofs).                                                 */
/* ------------------------------------------------------------------------------ */

/* dP = (d/dt) dW/dF(F + t dF) at t = 0.
 * Neo-Hookean, from dW/dF = C1 (2F - (2/det) cof) + 2 D1 (det - 1) cof with cof_jm =
 * ddet/dF_jm: d(det) = sum cof_jm dF_jm, d(cof_jm) = derivative of the same signed minor,
 *   dP = C1 (2 dF + (2/det^2) d(det) cof - (2/det) d(cof)) + 2 D1 (d(det) cof + (det - 1) d(cof)).
 * p-Laplacian, from dW/dF = s^((p-2)/2) F with s = |F|^2:
 *   dP = s^((p-2)/2) dF + (p - 2) s^((p-4)/2) (F . dF) F,
 * with dP = dF for p = 2 and dP = 0 at F = 0 otherwise (the Hessian of |F|^p / p is 0 there
 * for p > 2 and unbounded for p < 2). */
static void or_d2W(const or_mesh* M, double F[3][3], double dF[3][3], double dP[3][3], int* dom_err) {
    const int dim = M->dim;
    if (M->model == OR_NEOHOOKE) {
        double det = or_det(dim, F);
        if (!(det > 0.0)) *dom_err = 1;
        double cof[3][3], dcof[3][3], ddet = 0.0;
        for (int j = 0; j < dim; ++j)
            for (int m = 0; m < dim; ++m) {
                double minor, dminor;
                if (dim == 2) {
                    minor = F[1 - j][1 - m];
                    dminor = dF[1 - j][1 - m];
                } else {
                    int r[2], c[2], nr = 0, nc = 0;
                    for (int a = 0; a < 3; ++a) if (a != j) r[nr++] = a;
                    for (int a = 0; a < 3; ++a) if (a != m) c[nc++] = a;
                    minor = F[r[0]][c[0]] * F[r[1]][c[1]] - F[r[0]][c[1]] * F[r[1]][c[0]];
                    dminor = dF[r[0]][c[0]] * F[r[1]][c[1]] + F[r[0]][c[0]] * dF[r[1]][c[1]]
                           - dF[r[0]][c[1]] * F[r[1]][c[0]] - F[r[0]][c[1]] * dF[r[1]][c[0]];
                }
                int sgn = ((j + m) % 2 == 0) ? 1 : -1;
                cof[j][m] = sgn * minor;
                dcof[j][m] = sgn * dminor;
                ddet += cof[j][m] * dF[j][m];
            }
        for (int j = 0; j < dim; ++j)
            for (int m = 0; m < dim; ++m)
                dP[j][m] = M->C1 * (2.0 * dF[j][m] + (2.0 / (det * det)) * ddet * cof[j][m]
                                    - (2.0 / det) * dcof[j][m])
                         + 2.0 * M->D1 * (ddet * cof[j][m] + (det - 1.0) * dcof[j][m]);
        return;
    }
    if (M->model == OR_PLAPLACE_LP) {   /* dP_m = (p-1) |F_m|^(p-2) dF_m (dF_m for p = 2) */
        for (int m = 0; m < dim; ++m) {
            double c = (M->p == 2.0) ? 1.0 : (F[0][m] != 0.0) ? (M->p - 1.0) * pow(fabs(F[0][m]), M->p - 2.0) : 0.0;
            dP[0][m] = c * dF[0][m];
        }
        return;
    }
    double s = 0.0, fd = 0.0;
    for (int m = 0; m < dim; ++m) {
        s += F[0][m] * F[0][m];
        fd += F[0][m] * dF[0][m];
    }
    double c1, c2;
    if (M->p == 2.0) {
        c1 = 1.0;
        c2 = 0.0;
    } else if (s > 0.0) {
        c1 = pow(s, (M->p - 2.0) / 2.0);
        c2 = (M->p - 2.0) * pow(s, (M->p - 4.0) / 2.0);
    } else {
        c1 = c2 = 0.0;
    }
    for (int m = 0; m < dim; ++m) dP[0][m] = c1 * dF[0][m] + c2 * fd * F[0][m];
}

int or_hessian_vector(int model, double p, double C1, double D1, int dim, int d, int64_t nn,
                      const double* coords, int64_t ne, const int32_t* elems,
                      const double* dphi, const double* vol, const uint8_t* dirichlet,
                      const int64_t* row_ptr, const int64_t* ent, const double* v,
                      const double* w, double* Hw) {
    if (!or_check_model(model, dim, d)) return OR_EINVAL;
    or_mesh M = {model, dim, d, p, C1, D1, coords, elems, dphi, vol};
    const int k = dim + 1;
    double* r = (double*)malloc(sizeof(double) * (size_t)(ne > 0 ? ne * k * d : 1));
    if (!r) return OR_ENOMEM;
    int dom_err = 0;
    for (int64_t e = 0; e < ne; ++e) {
        double uloc[4][3], F[3][3], dF[3][3], dP[3][3];
        or_local_values(&M, e, v, uloc);
        or_element_F(&M, e, uloc, F);
        const int32_t* en = elems + e * k;
        const double* de = dphi + e * k * dim;
        for (int j = 0; j < d; ++j)
            for (int m = 0; m < dim; ++m) {
                double s = 0.0;
                for (int l = 0; l < k; ++l) {
                    int64_t n = (int64_t)en[l] * d + j;
                    double wl = (dirichlet && dirichlet[n]) ? 0.0 : w[n];
                    s += wl * de[l * dim + m];
                }
                dF[j][m] = s;
            }
        or_d2W(&M, F, dF, dP, &dom_err);
        for (int l = 0; l < k; ++l)
            for (int j = 0; j < d; ++j) {
                double s = 0.0;
                for (int m = 0; m < dim; ++m) s += dP[j][m] * de[l * dim + m];
                r[(e * k + l) * d + j] = vol[e] * s;
            }
    }
    for (int64_t i = 0; i < nn; ++i)
        for (int j = 0; j < d; ++j) {
            double s = 0.0;
            for (int64_t q = row_ptr[i]; q < row_ptr[i + 1]; ++q) s += r[ent[q] * d + j];
            int64_t n = i * d + j;
            Hw[n] = (dirichlet && dirichlet[n]) ? 0.0 : s;
        }
    free(r);
    return dom_err ? OR_EDOMAIN : OR_OK;
}
