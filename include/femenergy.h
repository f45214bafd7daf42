/*
 * femenergy.h -- C ABI of libfemenergy.so: evaluation of the discrete nonlinear energy
 * J(v) and its gradient over P1 triangles (dim = 2) and tetrahedra (dim = 3) on one
 * NVIDIA GB300 GPU (sm_103a).
 *
 * The method is that of Moskovka & Valdman, "Fast MATLAB evaluation of nonlinear
 * energies using FEM in 2D and 3D: Nodal elements" (arXiv 2109.01158):
 *   J(v) = J_grad(v) - b.v,   J_grad(v) = sum_k |T_k| W(grad v |T_k)        (eq. Denergy)
 *   b^(j) = M f^(j)  (P1 mass matrix M, nodal load f)                      (eqs. mass2D, linearTerm2)
 * with the compressible Neo-Hookean density (eq. neoHook) for the vector deformation v
 * (d = dim) or the p-Laplacian density (1/p)|grad v|^p (eq. pLaplacian, d = 1).
 *
 * Conventions shared by every entry point:
 *   - Indices are 0-based.  Node i has coordinates coords[i*dim + m] (the paper's
 *     nodes2coord); element e has nodes elems[e*(dim+1) + l] (elems2nodes, the map I_LG).
 *   - Degrees of freedom are interleaved as in Section 5 (eq. bvvectors): dof n = d*i + j is
 *     component j of node i.  v, g, f and the Dirichlet mask use this order, always in the
 *     caller's node numbering, whatever internal reordering the library applies.
 *   - Pointers named *_host are host memory; all other array pointers of the evaluation
 *     calls are DEVICE memory owned by the caller (e.g. torch tensors) on the context's
 *     device.  Host arrays passed to set-up calls are copied; the caller keeps ownership.
 *   - Evaluation calls are asynchronous on the context's stream.  Their return value
 *     reports argument and launch errors only; errors found on the device (an element with
 *     det F <= 0) are reported by fe_sync_status() or by the *_host calls.
 *   - No call throws; every call returns an fe_status.  fe_last_error() gives a message
 *     for the last failing call of the calling thread.
 *   - Results are deterministic: the same inputs give bitwise identical outputs run to
 *     run (no floating-point atomics; fixed reduction trees and patch-sum orders).
 */
#ifndef FEMENERGY_H
#define FEMENERGY_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fe_ctx fe_ctx; /* opaque; the library owns every mesh buffer on the device */

typedef enum {
    FE_OK = 0,
    FE_EINVAL = 1,   /* bad argument, malformed mesh, or call out of order              */
    FE_ENOMEM = 2,   /* device or host allocation failed                               */
    FE_ECUDA = 3,    /* CUDA runtime error (message in fe_last_error)                  */
    FE_EDOMAIN = 4,  /* Neo-Hookean: some element has det F <= 0; J = +Inf              */
    FE_ETIMEOUT = 5, /* a bounded device wait gave up                                  */
    FE_EBUSY = 6     /* resource in use                                                */
} fe_status;

/* FE_PLAPLACE: W = (1/p) |grad v|^p with the Euclidean norm, (1/p)(|grad v|^2)^(p/2).
 * FE_PLAPLACE_LP: W = (1/p) sum_m |dv/dx_m|^p, the same eq. pLaplacian read with the l^p norm
 * of the gradient (the two agree for p = 2); the minimal energies printed in the table of
 * Benchmark 6 are those of this reading.  Evaluated in FP64 only (not by the FE_DF64,
 * FE_F32_COMP, batched or no-allocation calls, which return FE_EINVAL for it). */
typedef enum { FE_PLAPLACE = 0, FE_NEOHOOKE = 1, FE_PLAPLACE_LP = 2 } fe_model;

/* Arithmetic of the element kernels (none is prescribed by the paper, which runs MATLAB
 * doubles).  FE_F64: IEEE double throughout.  FE_F32_COMP: per-element float arithmetic in
 * displacement form with double-precision patch sums and compensated double-precision energy
 * reductions; its error against the FP64 result is of float order (about 1e-7 relative).
 * FE_DF64: every per-element operation in double-float arithmetic (pairs of floats, about
 * 48 significand bits) on the FP32 pipes, with FP64 block and grid reductions; meets the
 * FP64 tolerances (energy 1e-12 of its condition number, gradient 1e-10 of its max norm)
 * for values within about 1e-30..1e30 in magnitude. */
typedef enum { FE_F64 = 0, FE_F32_COMP = 1, FE_DF64 = 2 } fe_precision;

/* Internal node/element numbering used for the device layout (invisible to callers).
 * FE_ORDER_MORTON sorts nodes along a Morton (Z-order) curve of their coordinates;
 * FE_ORDER_RCM is the reverse Cuthill-McKee numbering of the node graph (nodes adjacent when
 * they share an element), which keeps the index distance between neighbours small.  Both
 * then sort the elements by their least renumbered node. */
typedef enum { FE_ORDER_NONE = 0, FE_ORDER_MORTON = 1, FE_ORDER_RCM = 2 } fe_order;

/* Meaning of the vector v passed to the evaluation calls.  FE_INPUT_DEFORMATION: v is the
 * deformation (the paper's unknown, Sec. 3), v = X + u for the Neo-Hookean model.
 * FE_INPUT_DISPLACEMENT: v is the displacement u itself (Neo-Hookean only; the p-Laplacian
 * ignores it) -- same J and gradient, but small displacements keep their full relative
 * precision instead of being rounded to the spacing of doubles near X. */
typedef enum { FE_INPUT_DEFORMATION = 0, FE_INPUT_DISPLACEMENT = 1 } fe_input;

/* Numbering of the dof vectors of the evaluation calls.  FE_VECTORS_CALLER (default): the
 * caller's node numbering.  FE_VECTORS_DEVICE: the library's internal numbering (the
 * renumbering of FE_ORDER_MORTON or FE_ORDER_RCM; the same as the caller's with
 * FE_ORDER_NONE), which skips
 * the permutation on input and output -- for iterates that stay on the device. */
typedef enum { FE_VECTORS_CALLER = 0, FE_VECTORS_DEVICE = 1 } fe_vector_order;

/* Library version (major*10000 + minor*100 + patch). */
int fe_version(void);

/* Message describing the last failing call on this thread (owned by the library). */
const char* fe_last_error(void);

/* The node renumbering that fe_mesh_upload applies for `order`, computed on the host
 * (no context, no device work).  The mesh arguments are those of fe_mesh_upload and are
 * validated the same way.  perm_out (n_nodes int32, caller-owned) receives perm[new] = old:
 * the identity for FE_ORDER_NONE.  FE_EINVAL on a malformed mesh or a bad order. */
fe_status fe_node_order(int dim, int64_t n_nodes, const double* coords_host, int64_t n_elems,
                        const int32_t* elems_host, int order, int32_t* perm_out);

/* Create a context on CUDA device `device` that enqueues all work on `cuda_stream`
 * (a cudaStream_t; NULL = the legacy default stream).  *out receives the context. */
fe_status fe_create(fe_ctx** out, int device, void* cuda_stream);

/* Release every device and host buffer of the context (synchronises its stream). */
fe_status fe_destroy(fe_ctx* ctx);

/* Change the stream later calls enqueue on. */
fe_status fe_set_stream(fe_ctx* ctx, void* cuda_stream);

/* Upload a mesh (the paper's `mesh` structure, Sec. 4.1).
 *   dim        2 (triangles) or 3 (tetrahedra)
 *   d          components per node: 1 (scalar, p-Laplacian) or dim (Neo-Hookean)
 *   n_nodes    |N|;  coords_host: n_nodes*dim doubles, row-major (nodes2coord)
 *   n_elems    |T|;  elems_host:  n_elems*(dim+1) int32 node ids in [0, n_nodes)
 *   dirichlet_host: n_nodes*d bytes, 1 = fixed dof (dofsDirichlet), 0 = free (dofsMinim);
 *                   NULL = every dof free
 *   order      FE_ORDER_NONE keeps the caller's numbering; FE_ORDER_MORTON (Morton curve) and
 *              FE_ORDER_RCM (reverse Cuthill-McKee) renumber the nodes and sort elements by
 *              their first renumbered node so that the gathers of v hit L2
 * Validates ids and sizes (n_elems*(dim+1) < 2^31).  Replaces any previous mesh and
 * invalidates the precompute.  FE_EINVAL on a malformed mesh. */
fe_status fe_mesh_upload(fe_ctx* ctx, int dim, int d, int64_t n_nodes,
                         const double* coords_host, int64_t n_elems,
                         const int32_t* elems_host, const uint8_t* dirichlet_host,
                         int order);

/* Select the density: FE_PLAPLACE or FE_PLAPLACE_LP with exponent p > 1 (eq. pLaplacian;
 * requires d = 1),
 * or FE_NEOHOOKE with constants C1, D1 (eq. neoHook; requires d = dim).  For material
 * data, C1 = mu/2 and D1 = K/2 with mu = E/(2(1+nu)), K = E/(3(1-2nu)) (Benchmark 2). */
fe_status fe_set_model(fe_ctx* ctx, int model, double p, double C1, double D1);

/* Nodal load f in V_h (n_nodes*d doubles, host, dof order; NULL = 0).  The library forms
 * b = M f with the P1 mass matrix on the device at fe_precompute (eq. linearTerm2). */
fe_status fe_set_load(fe_ctx* ctx, const double* f_host);

/* Per-mesh precompute on the device (Sec. 4.1-4.2, done once per mesh): element volumes
 * |T| and shape-function gradients dphi, the nodal-patch CSR (node -> (element, local
 * index)) in increasing element order, b = M f, and the device buffers of the requested
 * precisions.  precisions: bit mask of 1 << FE_F64, 1 << FE_F32_COMP, 1 << FE_DF64.  The
 * active precision becomes FE_F64 if it is in the mask, else FE_DF64, else FE_F32_COMP;
 * fe_set_precision switches between precomputed ones.  The central-difference gradient needs
 * FE_F64.  FE_EINVAL if an element is degenerate. */
fe_status fe_precompute(fe_ctx* ctx, unsigned precisions);

/* Choose the arithmetic of later evaluation calls (must have been precomputed). */
fe_status fe_set_precision(fe_ctx* ctx, int precision);

/* Choose what the v argument of later evaluation calls (fe_energy ... fe_gradient_fd,
 * fe_energy_gradient_host and the batched calls on this mesh) means: FE_INPUT_DEFORMATION
 * (default) or FE_INPUT_DISPLACEMENT.  With displacements the energy is still
 * J = sum |T| W(I + grad u) - b.(X + u), with b.X formed once per load (Neumaier sum) and
 * b.u summed per call.  Any time after fe_create; FE_EINVAL for another value. */
fe_status fe_set_input(fe_ctx* ctx, int input);

/* Order of the dof vectors (fe_vector_order) of fe_energy, fe_gradient_exact,
 * fe_energy_gradient, fe_energy_gradient_host, fe_gradient_fd (also of its dof subset),
 * fe_hessian_vector and fe_cg_steihaug.  The batched calls and the server always use the
 * caller's order.  Any time after fe_create; FE_EINVAL for another value. */
fe_status fe_set_vector_order(fe_ctx* ctx, int order);

/* Permute a dof vector between the caller's numbering (x_dev) and the device numbering
 * (y_dev): y[d*i + j] = x[d*perm(i) + j] with perm the device -> caller node map of the
 * uploaded mesh.  n_nodes*d doubles each, device memory, on the context's stream; the two
 * must not overlap (FE_EINVAL if they are the same pointer).  Needs a mesh. */
fe_status fe_to_device_order(fe_ctx* ctx, const double* x_dev, double* y_dev);
fe_status fe_from_device_order(fe_ctx* ctx, const double* y_dev, double* x_dev);

/* Device bytes held by the context (mesh, precompute and work buffers). */
fe_status fe_footprint(const fe_ctx* ctx, size_t* bytes);

/* Energy (Sec. 5): *J_dev = sum_k |T_k| W(F_k) - b.v  (one double, device).
 *   v_dev    n_nodes*d doubles (device), full vector including Dirichlet values
 *   dens_dev NULL, or n_elems doubles (device) receiving W(F_k) per element (the paper's
 *            densities output), in the caller's element order
 * Neo-Hookean with some det F <= 0: *J_dev = +Inf and fe_sync_status returns FE_EDOMAIN. */
fe_status fe_energy(fe_ctx* ctx, const double* v_dev, double* J_dev, double* dens_dev);

/* Exact gradient (Sec. 6.2, eqs. dJdvn, dWFv): g_dev[n] = dJ/dv_n for every free dof n
 * (patch sum of |T| dW/dF : dF/dv_n, minus b_n) and 0 on Dirichlet dofs (Remark 1: the
 * gradient restricted to free dofs is g[free]).  g_dev: n_nodes*d doubles (device). */
fe_status fe_gradient_exact(fe_ctx* ctx, const double* v_dev, double* g_dev);

/* Energy and exact gradient in one pass over the elements (J_dev as in fe_energy). */
fe_status fe_energy_gradient(fe_ctx* ctx, const double* v_dev, double* J_dev, double* g_dev);

/* Hessian-vector product (not in the paper, whose trust-region solver uses the Hessian's
 * sparsity pattern only): Hw_dev = d/dt grad J(v + t w) at t = 0, the second derivative of
 * J_grad = sum_k |T_k| W(F_k) along w, gathered over the nodal patches like the exact
 * gradient (Sec. 6.2); b.v contributes nothing.  Entries of w_dev on Dirichlet dofs are
 * taken as 0 and the Dirichlet rows of Hw_dev are 0 (the Hessian on the free dofs).  v_dev,
 * w_dev, Hw_dev: n_nodes*d doubles (device, caller's dof order; v as set by fe_set_input).
 * p-Laplacian with p < 2: 0 where grad v = 0 (the Hessian is unbounded there).  Always
 * evaluated in FP64 (needs the FP64 precompute).  Neo-Hookean with some det F <= 0:
 * fe_sync_status returns FE_EDOMAIN. */
fe_status fe_hessian_vector(fe_ctx* ctx, const double* v_dev, const double* w_dev, double* Hw_dev);

/* Steihaug's truncated conjugate gradients (Nocedal & Wright, Alg. 7.2; not in the paper, the
 * inner solver of a trust-region Newton method like the one the paper minimises with, Sec. 7):
 * from z = 0, approximately minimises m(z) = g.z + z.H z / 2 over ||z||_2 <= radius, where H
 * is the Hessian of J at v on the free dofs (the product of fe_hessian_vector, FP64).  Stops
 * at the first of: ||g + H z||_2 <= tol; a direction d with d.H d <= 0, or a step that would
 * leave the ball (in both cases z moves along d to the boundary); max_cg products.
 *   v_dev      n_nodes*d doubles (device, caller's dof order): the point, as set by fe_set_input
 *   g_dev      n_nodes*d doubles (device): the gradient at v, 0 on Dirichlet dofs (as
 *              fe_gradient_exact returns it); not modified
 *   radius     > 0 and finite; tol >= 0 and finite; max_cg >= 0
 *   z_dev      n_nodes*d doubles (device, written): the step (0 on Dirichlet dofs)
 *   Hz_dev     n_nodes*d doubles (device, written): H z
 *   iters      host int (written): Hessian-vector products used; 0 when ||g|| <= tol already
 *   boundary   host int (written): 1 when z ended on the boundary, else 0
 * All vector work runs on the device (the dot products are fixed-order reductions, so the
 * results are bitwise reproducible); the call returns when the solve has finished.  Needs the
 * FP64 precompute; the first call allocates 3 vectors of n_nodes*d doubles of work space.
 * FE_EINVAL for a bad argument; Neo-Hookean with some det F <= 0 at v: fe_sync_status returns
 * FE_EDOMAIN and z is unspecified. */
fe_status fe_cg_steihaug(fe_ctx* ctx, const double* v_dev, const double* g_dev, double radius, double tol,
                         int max_cg, double* z_dev, double* Hz_dev, int* iters, int* boundary);

/* ---- L-BFGS memory on the device (not in the paper: the minimiser driven by the kernels) ----
 * The m most recent pairs s = v_new - v, y = g_new - g of a minimisation (oldest first) and
 * the direction d = -H g of the limited-memory BFGS inverse Hessian H, computed in the compact
 * representation of Byrd, Nocedal & Schnabel (1994, Thm. 2.2), with H_0 = (s.y / y.y) I of
 * the newest pair: the same H as the two-loop recursion (Nocedal & Wright, Alg. 7.4) in exact
 * arithmetic.  With no pairs, d = -g / ||g||.  Vectors are n doubles on the device; the
 * memory holds 2 (m + 1) n doubles.  Reductions are fixed-order: results are bitwise
 * reproducible.  Each call enqueues on the stream given at creation and returns once its
 * scalar is on the host. */
typedef struct fe_lbfgs fe_lbfgs;

/* n >= 1 unknowns, 1 <= m <= 16 pairs; stream: a cudaStream_t (NULL = legacy default). */
fe_status fe_lbfgs_create(fe_lbfgs** out, int device, void* stream, int64_t n, int m);
fe_status fe_lbfgs_destroy(fe_lbfgs* lb);
/* Forget every pair (the next direction is -g / ||g||). */
fe_status fe_lbfgs_reset(fe_lbfgs* lb);
/* Pairs in use (0..m). */
fe_status fe_lbfgs_pairs(const fe_lbfgs* lb, int* count);
/* Offer the pair s = v_new - v, y = g_new - g (device vectors of n doubles; not modified).
 * *sy (host) receives s.y; the pair is kept when s.y > 0, replacing the oldest one when m
 * pairs are held, and discarded otherwise. */
fe_status fe_lbfgs_update(fe_lbfgs* lb, const double* v_new_dev, const double* v_dev, const double* g_new_dev,
                          const double* g_dev, double* sy);
/* d_dev (n doubles, device, written) = -H g_dev; *gd (host) = g.d.  g_dev and d_dev must not
 * overlap. */
fe_status fe_lbfgs_direction(fe_lbfgs* lb, const double* g_dev, double* d_dev, double* gd);
/* One accepted L-BFGS step in one host round trip: fe_lbfgs_update with (v_new, v, g_new, g),
 * then fe_lbfgs_direction at g_new into d_dev, and max_i |g_new_i|.  out3 (host, 3 doubles)
 * receives s.y, g_new.d and max |g_new|.  The same pairs and direction as the two calls. */
fe_status fe_lbfgs_step(fe_lbfgs* lb, const double* v_new_dev, const double* v_dev, const double* g_new_dev,
                        const double* g_dev, double* d_dev, double* out3);
/* Checkpoint (not in the paper; its Benchmark 4 only warm-starts from the previous minimum):
 * copy the pairs in use, oldest first, to host memory -- s_host and y_host receive pair i at
 * [i*n, (i+1)*n), sy_host and yy_host the products s_i.y_j and y_i.y_j at [i*count + j] --
 * and *count the number of pairs.  Every buffer must hold m pairs (m*n, m*m doubles); the
 * buffers may be NULL when no pair is held.  Waits for the memory's stream. */
fe_status fe_lbfgs_save(const fe_lbfgs* lb, double* s_host, double* y_host, double* sy_host, double* yy_host,
                        int* count);
/* Resume: replace the memory of lb (created with the same n and an m >= count) by count saved
 * pairs and their products, as written by fe_lbfgs_save.  The directions and updates that
 * follow are bitwise those the saved memory would have given.  FE_EINVAL for count > m. */
fe_status fe_lbfgs_restore(fe_lbfgs* lb, const double* s_host, const double* y_host, const double* sy_host,
                           const double* yy_host, int count);

/* Central-difference gradient over nodal patches (Sec. 6.1, eqs. CD, CDS, jgradpm,
 * sumpatch): for dof n of node i, component j,
 *   g_n = ( sum_{T in T^i} |T| W(F_T^+) - sum_{T in T^i} |T| W(F_T^-) ) / (2 eps) - b_n,
 * where F_T^{+-} is F_T with row j recomputed from nodal values whose (i, j) entry is
 * shifted by +-eps (the paper's GG layers).  Dirichlet dofs give 0.
 *   dofs_dev NULL: every dof, g_dev has n_nodes*d entries.
 *   dofs_dev non-NULL: n_dofs int64 dof ids (device); g_dev[q] is the value for dofs_dev[q].
 * Always evaluated in FP64.  eps > 0. */
fe_status fe_gradient_fd(fe_ctx* ctx, const double* v_dev, double eps, double* g_dev,
                         const int64_t* dofs_dev, int64_t n_dofs);

/* End-to-end call with HOST buffers: evaluates the energy and the exact gradient of v_host
 * and returns J and g in host memory, then synchronises.  J_host: one double; g_host:
 * n_nodes*d doubles.  Page-locked buffers (cudaMallocHost / cudaHostAlloc, mapped into the
 * device address space) are read and written by the kernels directly over the host link;
 * pageable buffers are copied through device staging buffers.  Returns FE_EDOMAIN if some
 * det F <= 0. */
fe_status fe_energy_gradient_host(fe_ctx* ctx, const double* v_host, double* J_host,
                                  double* g_host);

/* Pipelined form of fe_energy_gradient_host for a sequence of evaluations: enqueues the
 * copy of v_host into one of two device slots (on a copy-in stream), the evaluation of J and
 * the exact gradient (on the context's stream) and the copies of J and g back to J_host and
 * g_host (on a copy-out stream), and returns without waiting.  Successive calls alternate
 * between the slots, so the copies of evaluation k + 1 in and of evaluation k - 1 out overlap
 * evaluation k.  Arguments as for fe_energy_gradient_host; the copies overlap only when the
 * host buffers are page-locked.  The caller keeps v_host unchanged, and reads J_host and
 * g_host, only after fe_host_wait.  The slots hold 2 (2 n_nodes d + 1) doubles of device
 * memory until the next fe_precompute, fe_mesh_upload or fe_destroy. */
fe_status fe_energy_gradient_host_async(fe_ctx* ctx, const double* v_host, double* J_host,
                                        double* g_host);

/* Wait until every evaluation enqueued by fe_energy_gradient_host_async has been copied
 * back; then as fe_sync_status (FE_EDOMAIN if any of them, or any other call since the last
 * status read, met det F <= 0). */
fe_status fe_host_wait(fe_ctx* ctx);

/* Watchdog of the device waits (failure detection; not in the paper).  The kernels that
 * stage data with bulk asynchronous copies wait for each copy at most `cycles` SM clocks
 * (0 = the default, 2e9, about one second) before they give up: the kernel then records
 * FE_ETIMEOUT (returned by the next fe_sync_status), waits with the default limit for the
 * copies it has in flight, and returns without finishing its outputs.  A short limit makes
 * that path run on purpose (tests of failure detection); the context stays usable and the
 * next call with the default limit is correct.  FE_EINVAL for cycles < 0. */
fe_status fe_set_wait_limit(fe_ctx* ctx, int64_t cycles);

/* Synchronise the stream and return (and clear) the device-side status of the calls
 * since the last fe_sync_status: FE_EDOMAIN if an element had det F <= 0, else FE_OK. */
fe_status fe_sync_status(fe_ctx* ctx);

/* Read back the precompute for inspection (synchronous, host outputs, caller's element
 * order): dphi_host[(e*(dim+1)+l)*dim + m] = d(phi_{e,l})/d(x_m), vol_host[e] = |T_e|. */
fe_status fe_get_shape_gradients(fe_ctx* ctx, double* dphi_host, double* vol_host);

/* Read back the nodal patches in the caller's numbering (synchronous): row_ptr_host has
 * n_nodes+1 entries, ent_host n_elems*(dim+1) entries e*(dim+1)+l, rows in increasing
 * element order (the offsets p_i of eq. pind1 and the patch rows of Sec. 4.2). */
fe_status fe_get_patches(fe_ctx* ctx, int64_t* row_ptr_host, int64_t* ent_host);

/* Read back b = M f in dof order (synchronous, host output of n_nodes*d doubles). */
fe_status fe_get_load_vector(fe_ctx* ctx, double* b_host);

/* Diagnostic: y_dev[i] = log(x_dev[i]) computed by the double-float logarithm of the
 * FE_DF64 kernels (x > 0, n doubles, device), so that its accuracy can be checked against a
 * reference logarithm.  Needs the FE_DF64 precompute. */
fe_status fe_diag_df64_log(fe_ctx* ctx, const double* x_dev, double* y_dev, int64_t n);

/* Number of kernels this context has launched since creation (instrumentation). */
fe_status fe_launch_count(const fe_ctx* ctx, int64_t* count);

/* Kernel timing (instrumentation).  While enabled, every kernel launch of the evaluation
 * calls is bracketed by a pair of CUDA events on the context stream, grouped by stage:
 *   0 node preparation, 1 element kernel, 2 patch gather, 3 central-difference element
 *   kernel, 4 central-difference gather / subset kernel.
 * fe_profile_read synchronises the stream, writes the summed milliseconds and the launch
 * count of each of the first n_stages stages (n_stages <= FE_PROFILE_STAGES) to host
 * arrays, and resets the sums. */
#define FE_PROFILE_STAGES 5
fe_status fe_profile_enable(fe_ctx* ctx, int enable);
fe_status fe_profile_read(fe_ctx* ctx, double* ms_host, int64_t* launches_host, int n_stages);


/* ---- Batched evaluation over many resident meshes (serving) -------------------------
 * Not in the paper: evaluates J and the exact gradient (same definitions as
 * fe_energy_gradient, double-float arithmetic as FE_DF64) for many independent requests,
 * each on its own precomputed mesh, in ONE persistent kernel launch whatever their number
 * (plus one host-to-device copy of the requests' descriptors).  The launch walks a work
 * list of 256-node and 256-element tiles of all requests in the order given; a tile that
 * needs the results of others of its request waits for them (bounded: see
 * fe_batch_set_wait_limit).  Every request's partial sums are reduced in an order fixed by
 * its own mesh, so its J and g are bitwise the same alone and in any mix of requests (they
 * can differ in the last bits from fe_energy_gradient, whose reduction tree is shaped by
 * the grid). */
typedef struct fe_batch fe_batch;

typedef struct {
    const fe_ctx* mesh; /* precomputed with FE_DF64 and given a model; only read              */
    const double* v;    /* n_nodes*d doubles (caller's dof order): device memory, or          */
                        /* page-locked host memory that the kernel reads directly             */
    double* J;          /* one double: device or page-locked host memory                      */
    double* g;          /* n_nodes*d doubles: device or page-locked host memory (written      */
                        /* directly by the kernel)                                            */
    void* work;         /* device scratch of fe_batch_work_bytes(mesh) bytes, 256-byte aligned;  */
                        /* owned by the caller, one per request in flight                       */
    int* done;          /* NULL, or an int (device or page-locked host memory) that the        */
                        /* kernel sets, once this request's J and g are written and visible to */
                        /* the host, to 1 (or 3 if one of its waits gave up: results invalid); */
                        /* the caller zeroes it before the call                                 */
} fe_batch_item;

/* Bytes of device scratch one request on `mesh` needs. */
fe_status fe_batch_work_bytes(const fe_ctx* mesh, size_t* bytes);
/* Create a batch executor on `device` enqueuing on `cuda_stream`. */
fe_status fe_batch_create(fe_batch** out, int device, void* cuda_stream);
fe_status fe_batch_destroy(fe_batch* b);
/* SM clocks a tile waits for the tiles it depends on before it gives up (then the request's
 * results are invalid and fe_batch_sync_status returns FE_ETIMEOUT); 0 restores the default
 * 2e9; negative is FE_EINVAL.  The waits end by construction (a tile only waits for tiles
 * handed out before it, to running blocks); the limit guards against a fault elsewhere. */
fe_status fe_batch_set_wait_limit(fe_batch* b, int64_t cycles);
/* Enqueue one evaluation of every item (asynchronous; the host descriptors are copied before
 * the call returns).  Items of one call must use distinct `work` buffers.  Neo-Hookean items
 * with some det F <= 0 get J = +Inf and fe_batch_sync_status returns FE_EDOMAIN. */
fe_status fe_batch_energy_gradient(fe_batch* b, const fe_batch_item* items, int n_items);
/* Synchronise the batch stream; FE_ETIMEOUT if a wait gave up, else FE_EDOMAIN if an item had
 * det F <= 0, since the last call. */
fe_status fe_batch_sync_status(fe_batch* b);
/* Kernel launches enqueued so far (one per non-empty fe_batch_energy_gradient call). */
fe_status fe_batch_launch_count(const fe_batch* b, int64_t* count);
/* The work list the batched kernel follows (host only, for inspection and tests): for n
 * requests with prep_tiles[k] node tiles and elem_tiles[k] element tiles (each >= 1) on a GPU
 * of resident_blocks resident blocks, the 3n ranges (request_out[q], step_out[q]: 0 prep,
 * 1 element, 2 gather) in list order, each starting at item start_out[q] and holding that
 * step's tiles; *total_out = the number of items.  Requests are grouped into waves of at
 * least 4 * resident_blocks tiles, pipelined as P(s), E(s-1), G(s-2). */
fe_status fe_batch_plan(int n, const int64_t* prep_tiles, const int64_t* elem_tiles, int64_t resident_blocks,
                        int64_t* start_out, int32_t* request_out, int32_t* step_out, int64_t* total_out);

/* ---- Continuous-batching server over resident meshes -------------------------------
 * Not in the paper: a native request loop around the persistent batched kernel.  Callers
 * submit energy + gradient requests (host vectors in, host results out); a worker thread
 * admits the requests that have arrived, in FIFO order, while their device scratch fits in
 * the HBM budget (a ring arena allocated at creation), orders the batch smallest mesh first
 * and enqueues it as one persistent launch on the server's own stream.  The kernel reads the
 * vectors and writes the gradients directly in page-locked host memory -- the caller's
 * buffers when they are page-locked (cudaMallocHost, cudaHostAlloc, cudaHostRegister),
 * otherwise the server's pinned staging (one extra host copy each way) -- and raises a
 * completion flag per request.  Batch k + 1 is prepared and enqueued while batch k runs; a
 * completion thread polls the flags and completes each request as soon as its own flag is
 * up (stamping its completion time), frees a batch's arena region once all its requests
 * are complete.  With max_batch > 1 the (up to three) batches in flight run on streams of
 * their own, so a batch starts on the SMs its predecessor frees during its last tiles; with
 * max_batch = 1 it serves one request at a time, in order on one stream, with the same
 * kernel.
 * Results are bitwise those of fe_batch_energy_gradient on the same request (alone or in
 * any mix).  Times are seconds on a steady clock since fe_server_create. */
typedef struct fe_server fe_server;

/* hbm_budget: bytes of device memory for the scratch of the in-flight requests;
 * max_batch >= 1: most requests per batch.  Creates its own non-blocking stream on `device`
 * and allocates everything it serves with up front: the arena, and per batch slot pinned
 * staging of min(max(hbm_budget/16, 1 MB), 256 MB) bytes for each direction (pageable
 * vectors also bound a batch by it; a single larger request grows it). */
fe_status fe_server_create(fe_server** out, int device, size_t hbm_budget, int max_batch);
/* Serve every submitted request, then stop the threads and free everything. */
fe_status fe_server_destroy(fe_server* s);
/* Queue one request.  mesh: precomputed with FE_DF64 and given a model (only read; it must
 * outlive the request).  v_host: n_nodes*d doubles, read when the request is admitted (keep
 * it unchanged until then).  J_host (one double) and g_host (n_nodes*d doubles) receive the
 * results at completion.  t_arrival: when the request arrives (server clock; < 0 = now);
 * arrivals must be submitted in non-decreasing order.  *ticket identifies it.  FE_EINVAL if
 * its device scratch exceeds the whole budget. */
fe_status fe_server_submit(fe_server* s, const fe_ctx* mesh, const double* v_host, double* J_host,
                           double* g_host, double t_arrival, int64_t* ticket);
/* Block until request `ticket` completed; returns its status (FE_OK; FE_EDOMAIN when some
 * det F <= 0 and J = +Inf; FE_ETIMEOUT or FE_ECUDA when the device failed it) and its
 * arrival, start (batch enqueued) and completion times (any pointer may be NULL).  Each
 * ticket can be waited for once. */
fe_status fe_server_wait(fe_server* s, int64_t ticket, double* t_arrival, double* t_start, double* t_done);
/* Seconds since fe_server_create on the server clock. */
fe_status fe_server_now(const fe_server* s, double* t);
/* Counters since creation: batches launched, largest batch, kernel launches, requests done. */
fe_status fe_server_stats(const fe_server* s, int64_t* batches, int64_t* max_batch, int64_t* launches,
                          int64_t* completed);
/* Zero those counters (e.g. between measurement runs). */
fe_status fe_server_reset_stats(fe_server* s);

/* ---- Device characterisation -------------------------------------------------------
 * Not in the paper: the issue rate of the FP64 unit, the roof of the FP64 kernels (bound by
 * FP64 arithmetic).  Runs eight independent chains of one operation per thread, four
 * 256-thread blocks per SM, 2^12 iterations (two launches of about 10 ms), and
 * returns operations per SM clock per SM (*per_clock_per_sm, from the SM cycle counter of
 * every block) and the SM clock the launch ran at in GHz (*sm_ghz, from the cycles and the
 * event time; may be NULL).  op: FE_RATE_DFMA, FE_RATE_DADD or FE_RATE_DMUL; anything else
 * is FE_EINVAL. */
enum { FE_RATE_DFMA = 0, FE_RATE_DADD = 1, FE_RATE_DMUL = 2 };
fe_status fe_fp64_rate(int device, int op, double* per_clock_per_sm, double* sm_ghz);

/* ---- Bounds-checking build ----------------------------------------------------------
 * Not in the paper: a debugging aid in place of a memory checker.  The library built with
 * -DFE_DEBUG_BOUNDS (libfemenergy_bounds.so; the Python package builds it with
 * build.build(bounds=True)) checks, in its kernels, every index read from memory before it
 * addresses another buffer: node ids of elements and tile records, CSR slots and rows,
 * local ids and slots of the FP32 tiles, caller node and element indices.  An index out of
 * range is not used (the access goes to entry 0 instead) and the first one is recorded with
 * the site that saw it (the BoundsSite numbers of csrc/bounds.cuh); no kernel traps.  In the
 * ordinary build the checks are not compiled in.
 *
 * fe_debug_bounds_enabled: 1 in the bounds-checking build, 0 otherwise.
 * fe_debug_bounds: reads and clears the record of `device` (waits for nothing: synchronise
 *   first); *site = 0 when nothing was out of range, else the site and *index the index.  In
 *   the ordinary build always *site = 0.
 * fe_debug_bounds_selftest: one checked read of entry `index` of a device buffer of n
 *   doubles (1 <= n <= 1024), so that an index outside [0, n) is recorded with site 99;
 *   synchronises the device.  FE_EINVAL in the ordinary build (the read would not be
 *   checked). */
int fe_debug_bounds_enabled(void);
fe_status fe_debug_bounds(int device, int* site, int64_t* index);
fe_status fe_debug_bounds_selftest(int device, int64_t index, int64_t n);

/* Energy without any allocation (the paper has no counterpart: this is an interface for
 * callers that cannot let this library allocate device memory -- a host program whose GPU
 * memory is owned entirely by its own pool allocator, or one whose time-critical loop must
 * not call cudaMalloc, which can synchronise the device).  It evaluates the same
 * J = sum_k |T_k| W(F_k) - b.v as fe_energy, with W in the same displacement form as the
 * context kernels (full relative accuracy near F = I), needs no context and no
 * fe_precompute, and calls no cudaMalloc, cudaFree or other allocating routine.
 *   device, cuda_stream   the device holding every array, and the stream to enqueue on
 *   dim, d, model, p, C1, D1   as in fe_mesh_upload / fe_set_model: FE_NEOHOOKE (d = dim),
 *               FE_PLAPLACE or FE_PLAPLACE_LP (d = 1, p > 1); anything else is FE_EINVAL
 *   coords_dev  n_nodes*dim doubles;  elems_dev  n_elems*(dim+1) int32 node ids, each in
 *               [0, n_nodes) (caller layouts of fe_mesh_upload, on the device)
 *   dphi_dev    n_elems*(dim+1)*dim doubles, vol_dev n_elems doubles: the shape gradients
 *               and volumes in the layout fe_get_shape_gradients returns
 *   b_dev       NULL (no load) or n_nodes*d doubles (b = M f);  v_dev  n_nodes*d doubles
 *   J_dev       one double receiving J: +Inf if some det F <= 0 (whatever the element's
 *               volume); NaN if some element names a node outside [0, n_nodes) (such an
 *               element is skipped without reading memory through its ids)
 * The arrays are only checked on the device, so those two outcomes arrive in J_dev, not in
 * the return status.  Its only scratch (block partial sums, a ticket and a flag word,
 * 19,472 bytes) is a static device array that every GPU loading the library keeps until the
 * process exits.  The first call on a device looks up that array's address; make it before
 * any stream capture.  All calls share the array: calls that overlap on the GPU race and
 * must be serialised by the caller.  Sizes beyond the maximum (n_elems*(dim+1) >= 2^31 or
 * n_nodes*d >= 2^31) and a device index that does not exist are rejected with FE_EINVAL. */
fe_status fe_energy_noalloc(int device, void* cuda_stream, int dim, int d, int model, double p,
                            double C1, double D1, int64_t n_nodes, const double* coords_dev,
                            int64_t n_elems, const int32_t* elems_dev, const double* dphi_dev,
                            const double* vol_dev, const double* b_dev, const double* v_dev,
                            double* J_dev);
#ifdef __cplusplus
}
#endif
#endif /* FEMENERGY_H */
