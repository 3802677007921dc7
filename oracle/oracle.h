/*
 * Plain FP64 CPU oracle for the energy-based FEM hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  It shares no code,
 * header, table or helper with the CUDA path under paper_2602_12365_b300/.
 *
 * What it computes (arXiv 2602.12365):
 *   Psi_h(u) = sum_e sum_q psi(grad u_h^e(xi_q)) w_q det J^e(xi_q)      (Eq. 2)
 *   r(u)     = grad Psi_h(u)                                           (Eq. 1)
 *   K(u) v   = directional derivative of r along v (the JVP of r)      (Eq. 3)
 * evaluated element by element in natural order as in Algorithm 1
 * (gather, field gradient, density, integrate, accumulate), with the
 * compressible Neo-Hookean density
 *   psi(F) = mu/2 (I1 - 3) - mu ln J + lambda/2 (ln J)^2,
 *   I1 = tr(F^T F) (+1 in 2D plane strain, F33 = 1),  J = det F.
 * Dirichlet conditions follow the condensation of Sec. 6.1: prescribed
 * components carry their values in u and are removed from r and K by a mask.
 *
 * Element types: 0 = P1 triangle (1 point, w = 1/2), 1 = P1 tetrahedron
 * (1 point, w = 1/6), 2 = Q1 hexahedron (2x2x2 Gauss, w = 1, VTK order).
 *
 * Layouts: X[n_nodes*dim], conn[n_el*n_en] (int32), mu/lam[n_el],
 * u/v/r/y[n_nodes*dim] node-major interleaved, mask[n_nodes*dim] (1 =
 * prescribed), D[n_nodes*dim*dim] row-major blocks.
 *
 * Status: 0 = ok, 3 = some J <= 0 (energy is +inf), 4 = non-finite input.
 */
#ifndef FEM_ORACLE_H
#define FEM_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

int ora_n_en(int etype);
int ora_dim(int etype);

/* psi, P = dpsi/dF, dP = (d^2 psi/dF^2) : dF for one deformation gradient */
double ora_nh_psi(int dim, const double* F, double mu, double lam);
void ora_nh_P(int dim, const double* F, double mu, double lam, double* P);
void ora_nh_dP(int dim, const double* F, const double* dF, double mu, double lam, double* dP);

/* Per-element geometry at quadrature point q: gradN[n_en*dim], returns w*detJ */
double ora_geometry(int etype, const double* Xe, int q, double* gradN, double* detJ);
int ora_n_qp(int etype);

/* Total energy (Neumaier-compensated sum of element energies, element
 * order).  psi_e (nullable) receives each element's energy; abs_sum
 * (nullable) receives the roundoff scale S = sum_e sum_q w detJ
 * (mu/2 I1 + mu |ln J| + lam/2 (ln J)^2). */
double ora_energy(int etype, int64_t n_nodes, int64_t n_el, const double* X,
                  const int32_t* conn, const double* mu, const double* lam,
                  const double* u, double* psi_e, double* abs_sum, int* status);

/* r = mask_out(grad Psi); mask may be NULL (no masking). */
void ora_residual(int etype, int64_t n_nodes, int64_t n_el, const double* X,
                  const int32_t* conn, const double* mu, const double* lam,
                  const double* u, const uint8_t* mask, int mask_out, double* r,
                  int* status);

/* y = Mo K(u) Mi v, Mi = mask on input if mask_in, Mo if mask_out. */
void ora_hvp(int etype, int64_t n_nodes, int64_t n_el, const double* X,
             const int32_t* conn, const double* mu, const double* lam,
             const double* u, const double* v, const uint8_t* mask, int mask_in,
             int mask_out, double* y, int* status);

/* Nodal diagonal blocks D_i = K_ii (dim x dim); prescribed components get an
 * identity row/column. */
void ora_block_diag(int etype, int64_t n_nodes, int64_t n_el, const double* X,
                    const int32_t* conn, const double* mu, const double* lam,
                    const double* u, const uint8_t* mask, double* D, int* status);

/* Per-element parameter VJP: g_mu[e] = a^T dr_e/dmu_e, g_lam[e] = a^T dr_e/dlam_e */
void ora_param_vjp(int etype, int64_t n_nodes, int64_t n_el, const double* X,
                   const int32_t* conn, const double* mu, const double* lam,
                   const double* u, const double* a, double* g_mu, double* g_lam,
                   int* status);

/* Newton-CG load stepping (one shared algorithm; see oracle.c). */
typedef struct {
    double newton_rtol;     /* 1e-8 */
    int newton_max;         /* 50 */
    double eta_max;         /* 0.1 */
    int cg_max;             /* 0 -> 10 * n_dofs */
    double predictor_rtol;  /* 1e-2 */
    double armijo_c;        /* 1e-4 */
    int ls_max;             /* 20 */
    double ls_eps;          /* roundoff guard epsilon, 2^-52 */
    int max_bisect;         /* 5 */
} ora_newton_opts;

typedef struct {
    int status;
    int newton_iters;
    int cg_iters;
    int bisections;
    double r0_norm;
    double r_norm;
    int ls_halvings;
} ora_newton_stats;

void ora_default_opts(ora_newton_opts* o);

/* Advance u (prescribed entries at s_prev*ubar on entry) to load factor s. */
int ora_load_step(int etype, int64_t n_nodes, int64_t n_el, const double* X,
                  const int32_t* conn, const double* mu, const double* lam,
                  const uint8_t* mask, const double* ubar, double s_prev, double s,
                  double* u, const ora_newton_opts* opts, ora_newton_stats* stats);

/* Per-node MLP y = W3 act(W2 act(W1 x + b1) + b2) + b3, FP64, row-major
 * W[out][in]; act = SiLU. */
void ora_mlp_forward(int n, int d_in, int h1, int h2, int d_out, const double* x,
                     const double* W1, const double* b1, const double* W2,
                     const double* b2, const double* W3, const double* b3,
                     double* y);
/* Given dL/dy, accumulate parameter gradients (gW*, gb*) and return dL/dx
 * (nullable). */
void ora_mlp_backward(int n, int d_in, int h1, int h2, int d_out, const double* x,
                      const double* W1, const double* b1, const double* W2,
                      const double* b2, const double* W3, const double* b3,
                      const double* gy, double* gW1, double* gb1, double* gW2,
                      double* gb2, double* gW3, double* gb3, double* gx);

/* Learned block preconditioner (3D).  Node graph: the distinct nodes that
 * share an element with node i (CSR; idx may be NULL to count).  Returns the
 * number of entries. */
int64_t ora_node_graph(int64_t nn, int64_t ne, int n_en, const int32_t* conn, int64_t* ptr,
                       int32_t* idx, int64_t cap);
/* 36 features per node from the nodal diagonal blocks D [nn*9] (identity on
 * prescribed components), the moduli and the per-DOF mask; the 27 block
 * features are compressed as sign(x) ln(1 + |x|). */
void ora_lp_features(int etype, int64_t nn, int64_t ne, const int32_t* conn, const double* mu,
                     const double* lam, const uint8_t* mask, const double* D, double* F);
/* M_i = F A A^T F^T / s_i from the 6 network outputs per node (see oracle.c);
 * returns 0 if some D_i is not SPD (that block is set to the identity). */
int ora_lp_blocks(int64_t nn, const double* D, const uint8_t* mask, const double* o, double* M);
/* dL/do from dL/dM. */
void ora_lp_blocks_backward(int64_t nn, const double* D, const uint8_t* mask, const double* o,
                            const double* gM, double* go);

/* Neural constitutive model (Sec. "Neural Constitutive Modeling"):
 *   psi = [NN(I1, J) - NN(3, 1)] + psi_NH,
 * NN: 2 -> H -> H -> 1 MLP, softplus activations, of I1 = tr(F^T F) (+1 in
 * plane strain) and J = det F.  params (H*H + 5H + 1 doubles): W1 [H][2],
 * b1 [H], W2 [H][H] (row m: unit m of layer 2), b2 [H], w3 [H], b3.
 * ora_ncm_set installs it for every element loop (energy, residual, HVP,
 * block diagonal, load step); H = 0 restores the Neo-Hookean law alone. */
int ora_ncm_set(int H, const double* params);
/* NN value, gradient [2] and Hessian [2][2] in (I1, J) (each nullable). */
void ora_ncm_eval(double I1, double J, double* y, double* g, double* h);
/* the point-level law as the element loops use it */
double ora_law_psi(int d, const double* F, double mu, double lam);
void ora_law_P(int d, const double* F, double mu, double lam, double* P);
void ora_law_dP(int d, const double* F, const double* dF, double mu, double lam, double* dP);

/* Sparse K by colouring (Sec. 2.2, Algorithm 2; App. A, B).
 * DOF pattern (App. B): CSR over DOFs (dof = node*dim + component), entry
 * (i, j) when the nodes of i and j share an element (the node itself
 * included), ascending columns; idx may be NULL to count.  Returns nnz. */
int64_t ora_dof_pattern(int64_t nn, int d, int64_t ne, int n_en, const int32_t* conn,
                        int64_t* ptr, int32_t* idx, int64_t cap);
/* Greedy distance-2 colouring of the columns in ascending order (App. A);
 * returns the number of colours. */
int ora_distance2_colors(int64_t n, const int64_t* ptr, const int32_t* idx, int32_t* colors);
/* K values on the pattern from K e_j = ora_hvp(e_j) for every column j
 * (masking as ora_hvp); returns 5 if some K e_j leaves the pattern. */
int ora_sparse_values(int etype, int64_t n_nodes, int64_t n_el, const double* X,
                      const int32_t* conn, const double* mu, const double* lam,
                      const double* u, const uint8_t* mask, int mask_in, int mask_out,
                      const int64_t* ptr, const int32_t* idx, double* vals, int* status);

#ifdef __cplusplus
}
#endif
#endif
