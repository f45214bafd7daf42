// fe_internal.cuh -- device layout, context and kernel entry points shared by the
// translation units of libfemenergy.so.  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <math_constants.h>
#include <stdint.h>

#include <atomic>
#include <string>
#include <vector>

#include "bounds.cuh"
#include "df64.cuh"
#include "femenergy.h"

namespace fe {

// Fixed launch shapes.  The element and node reductions use a grid that depends only on
// the problem size (never on the device), so every run sums the same partials in the same
// order and results are bitwise reproducible.
constexpr int kThreads = 256;
constexpr int kMaxElemBlocks = 2432;  // 16 x 152 SMs
constexpr int kMaxNodeBlocks = 608;   // 4 x 152 SMs

// Device status bits (accumulated until fe_sync_status).
constexpr int kStatusDomain = 1;      // det F <= 0 seen
constexpr int kStatusDegenerate = 2;  // |T| == 0 at precompute
constexpr int kStatusTimeout = 4;     // a bounded device wait gave up

// Model parameters passed by value to the element kernels.
struct ModelParams {
  double p, C1, D1;
  double twoC1, twoD1;   // 2 C1 and 2 D1
  int pcase;  // p-Laplacian: 2 -> p == 2, 3 -> p == 3, 0 -> general pow
  int64_t nn;  // nodes of the mesh (the bound of the node-id checks of the bounds-checking build)
};

inline int grid_for(int64_t n, int max_blocks) {
  int64_t b = (n + kThreads - 1) / kThreads;
  if (b < 1) b = 1;
  return (int)(b < max_blocks ? b : max_blocks);
}

// Element tiles of the fused element + patch kernels (fe_tiles.cu): a tile is a contiguous
// range of at most kTileElems device-order elements together with the nodes they touch (at
// most tile_max_nodes(dim)); the fused kernels run blocks of kTileThreads threads.
constexpr int kTileElems = 768;      // 128 hexahedra of six tetrahedra: one octree cell
constexpr int kTileNodeWarps = 3;    // warps that gather nodal values and sum patches
constexpr int kTileThreads = kTileElems + 32 * kTileNodeWarps + 32;   // + one producer warp
constexpr int tile_max_nodes(int dim) { return dim == 3 ? 256 : 512; }
// Tiles start on multiples of kTileAlign elements.
constexpr int kTileAlign = 4;
inline int64_t padded_ne(int64_t ne) { return (ne + kTileAlign - 1) / kTileAlign * kTileAlign; }

// Padded stride (in components) of the per-node displacement buffer: 1, 2 or 4.
inline int padded_d(int d) { return d == 3 ? 4 : d; }

// Scalars of the device-resident conjugate-gradient solver (fe_cg.cu).
struct CgState {
  double rr;       // r.r of the current residual
  double rrn;      // r.r after the last step
  double dd, zd, zz;  // d.d, z.d, z.z of the current direction and iterate
  double dHd;      // d.H d
  double radius2;  // squared trust-region radius
  double tol;      // stop at ||r|| <= tol
  int k;           // Hessian-vector products used
  int done;        // 1 once the solve has stopped
  int boundary;    // 1 if it stopped on the boundary
  int max_cg;
};

}  // namespace fe

// Context: all device buffers are in the internal ("device") numbering.
struct fe_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;

  // mesh
  int dim = 0, d = 0, order = 0;
  int64_t nn = 0, ne = 0;
  bool have_mesh = false, have_pre = false;
  unsigned pre_mask = 0;
  int precision = FE_F64;
  int model = FE_NEOHOOKE;
  double p = 2.0, C1 = 0.0, D1 = 0.0;
  bool model_set = false;
  int input = FE_INPUT_DEFORMATION;  // meaning of the v argument of the evaluation calls
  int vector_order = FE_VECTORS_CALLER;  // numbering of the dof vectors of the evaluation calls
  double bX = 0.0;              // b.X (Neo-Hookean), added to b.u when v is a displacement
  std::vector<double> f_host;   // load in the caller's dof order (empty = 0)
  std::vector<int32_t> perm_h;  // device node -> caller node (empty = identity)
  std::vector<int32_t> eperm_h; // device element -> caller element (empty = identity)

  // device: mesh
  double* X = nullptr;         // nn*dim, device node order
  int32_t* elems = nullptr;    // (dim+1) SoA arrays of ne node ids
  uint8_t* dir = nullptr;      // nn*d Dirichlet mask, device order
  int32_t* perm = nullptr;     // nn (null = identity)
  int32_t* iperm = nullptr;    // nn: caller node -> device node (null = identity)
  int32_t* eperm = nullptr;    // ne (null = identity)

  // device: precompute
  double* dphi = nullptr;      // dim*dim SoA arrays of ne: index (l-1)*dim + m, l = 1..dim
  double* vol = nullptr;       // ne
  int32_t* row_ptr = nullptr;  // nn+1
  int32_t* ent = nullptr;      // ne*(dim+1): e*(dim+1)+l, rows in increasing element order
  int32_t* slot = nullptr;     // (dim+1) SoA arrays of ne: CSR position of (e, l)
  double* b = nullptr;         // nn*d, device order
  // FP32 element data of the tiles (fe_eval_f32.cu): one block of tile_block_bytes_f32(dim)
  // bytes per tile, holding the tile's dphi, vol and tile_elem entries, so that one bulk copy
  // stages a tile
  unsigned char* blk32 = nullptr;
  float2* dphi_df = nullptr;   // double-float copy of dphi (hi, lo)
  float2* vol_df = nullptr;    // double-float copy of vol
  fe::LogEntry* log_tab = nullptr;  // table of the double-float logarithm

  // device: work buffers
  double* u = nullptr;         // nn*padded_d(d): displacement (Neo-Hookean) or v
  double* w_hvp = nullptr;     // nn*padded_d(d): direction of a Hessian-vector product
  double* r = nullptr;         // ne*(dim+1)*d slot-ordered local forces (x2 for FD)
  float2* u_df = nullptr;      // nn*padded_d(d) displacement as float pairs (FE_DF64, FE_F32_COMP)
  float2* r_df = nullptr;      // ne*(dim+1)*d double-float local forces
  double* partials = nullptr;  // element partials [kMaxElemBlocks] then node partials
  unsigned* counter = nullptr; // last-block ticket
  int* status = nullptr;       // device status bits
  double* stage_v = nullptr;   // staging for the *_host call
  double* stage_g = nullptr;
  double* stage_J = nullptr;
  // pipelined host evaluations (fe_energy_gradient_host_async): two device slots, a copy-in
  // and a copy-out stream, and per slot the events "copied in", "evaluated", "copied out"
  double* pipe_v[2] = {nullptr, nullptr};
  double* pipe_g[2] = {nullptr, nullptr};
  double* pipe_J = nullptr;    // 2 doubles, one per slot
  cudaStream_t pipe_in = nullptr, pipe_out = nullptr;
  cudaEvent_t pipe_ev[3][2] = {};
  int64_t pipe_k = 0;          // evaluations enqueued since the slots were allocated
  double* hvp_cache = nullptr; // per-element terms of the Hessian at the CG solver's point
  double* cg_vec = nullptr;    // 3*nn*d: residual, direction and H direction of the CG solver
  double* cg_part = nullptr;   // 2*kMaxNodeBlocks partial sums of the CG solver
  unsigned* cg_ticket = nullptr;  // last-block ticket of the CG solver
  fe::CgState* cg_state = nullptr;  // device scalars of the CG solver
  fe::CgState* cg_host = nullptr;   // page-locked host copy of them

  // device: element tiles (fe_tiles.cu).  Tile t holds the elements [tile_ebeg[t],
  // tile_ebeg[t+1]) and the tile nodes [tile_nbeg[t], tile_nbeg[t+1]) (sorted by node id).
  // tile_node[k] = {device node id i, caller node id perm[i], first local slot | slot count
  // << 16, (partial slot + 1) << 1 | owner}: partial slot -1 when every element of the node's
  // patch is in this tile, owner = 1 when this tile adds the node's b_i v_i;
  // tile_elem[e] = local node ids and local slots of element e (16 bits each: ids in .x/.y,
  // slots in .z/.w).  A node whose patch spans several tiles ("shared") receives one partial
  // sum per tile: the s-th shared node tile_snode[s] has the partial slots
  // tile_spart[tile_sbeg[s] .. tile_sbeg[s+1]) of tile_part.
  int64_t n_tiles = 0, n_tnodes = 0, n_shared = 0, n_tpart = 0;
  int32_t* tile_ebeg = nullptr;   // n_tiles + 1
  int32_t* tile_nbeg = nullptr;   // n_tiles + 1
  int4* tile_node = nullptr;      // n_tnodes
  uint4* tile_elem = nullptr;     // ne
  int32_t* tile_snode = nullptr;  // n_shared
  int32_t* tile_sbeg = nullptr;   // n_shared + 1
  int32_t* tile_spart = nullptr;  // n_tpart: partial slots of each shared node, in tile order
  float2* tile_part = nullptr;    // n_tpart * d: partial patch sums of the shared nodes
  double* tile_epart = nullptr;   // 2 * n_tiles: per-tile sums of |T| W (and of b.v)
  double* tile_bvp = nullptr;     // ceil(nn / kThreads): block partials of b.v of the node prep

  // SM clocks a bulk-copy kernel waits for its first copy before it gives up and reports
  // FE_ETIMEOUT (fe_set_wait_limit); the drain after giving up always waits the full default
  long long wait_limit = 2000000000LL;

  int64_t launches = 0;
  size_t bytes = 0;

  // kernel timing: per stage, a pool of event pairs recorded around each launch
  bool prof = false;
  std::vector<cudaEvent_t> prof_ev[FE_PROFILE_STAGES];
  int prof_n[FE_PROFILE_STAGES] = {0};
};

// True when the v argument of an evaluation is the Neo-Hookean displacement u = v - X.
inline bool input_is_disp(const fe_ctx* c) {
  return c->model == FE_NEOHOOKE && c->input == FE_INPUT_DISPLACEMENT;
}

// The permutation (device node -> caller node) applied to the dof vectors of the evaluation
// calls: the mesh's, or none when the caller works in the device numbering.
inline const int32_t* io_perm(const fe_ctx* c) {
  return c->vector_order == FE_VECTORS_DEVICE ? nullptr : c->perm;
}


namespace fe {

// error reporting (thread-local message)
fe_status set_error(fe_status st, const std::string& msg);
fe_status cuda_check(cudaError_t e, const char* what);

// fe_precompute.cu
// fe_batch.cu: the descriptor block and the persistent launch of the batched kernel (FE_DF64
// meshes).  host_stage (pinned) and dev_stage hold batch_stage_bytes(n) bytes (16-byte
// aligned); work buffers hold batch_work_bytes(mesh) bytes, 256-byte aligned.  One copy of
// the block and one launch on stream s; wait_limit (SM clocks, <= 0 = the default 2e9)
// bounds each wait of a tile for the tiles it depends on.
size_t batch_stage_bytes(int n);
size_t batch_work_bytes(const fe_ctx* m);
fe_status batch_enqueue(cudaStream_t s, int device, const fe_batch_item* items, int n, void* host_stage,
                        void* dev_stage, int* status, long long wait_limit);

// fe_eval_f64.cu / fe_hessian.cu
fe_status launch_node_prep_f64(fe_ctx* c, const double* v);
fe_status launch_hvp_f64(fe_ctx* c, const double* v, const double* w, double* Hw);
// The product along w at the v last prepared by launch_node_prep_f64 (c->u); does nothing
// when skip (nullable device flag) is nonzero.
fe_status launch_hvp_dir_f64(fe_ctx* c, const double* w, double* Hw, const int* skip);
// Products at a fixed point: prepare stores the v-dependent per-element terms in c->hvp_cache
// (hvp_cache_doubles(c) doubles); cached computes Hw from them, bitwise as launch_hvp_f64.
size_t hvp_cache_doubles(const fe_ctx* c);
fe_status launch_hvp_prepare_f64(fe_ctx* c, const double* v);
fe_status launch_hvp_cached_f64(fe_ctx* c, const double* w, double* Hw, const int* skip);
// fe_cg.cu: Steihaug's CG on the device (buffers cg_* allocated by the caller).
fe_status launch_cg_steihaug(fe_ctx* c, const double* v, const double* g, double radius, double tol, int max_cg,
                             double* z, double* Hz, int* iters, int* boundary);

fe_status launch_precompute(fe_ctx* c);
fe_status launch_load_vector(fe_ctx* c);

// fe_eval_f64.cu
fe_status launch_eval_f64(fe_ctx* c, const double* v, double* J, double* dens, double* g,
                          bool want_energy, bool want_grad);
fe_status launch_fd_f64(fe_ctx* c, const double* v, double eps, double* g,
                        const int64_t* dofs, int64_t ndofs);
fe_status launch_expand_dphi(fe_ctx* c, double* dphi_full, double* vol_user);

// fe_eval_df64.cu
fe_status launch_precompute_df(fe_ctx* c);
fe_status launch_eval_df64(fe_ctx* c, const double* v, double* J, double* dens, double* g,
                           bool want_energy, bool want_grad);
fe_status launch_diag_df_log(const LogEntry* tab, const double* x, double* y, int64_t n, cudaStream_t s);

// fe_eval_f32.cu
fe_status launch_eval_f32(fe_ctx* c, const double* v, double* J, double* dens, double* g,
                          bool want_energy, bool want_grad);

ModelParams model_params(const fe_ctx* c);

// Device allocation rounded up to 256 bytes plus 256 bytes of slack: bulk copies read whole
// 16-byte units, so a range that ends inside the last unit of a buffer stays in bounds.
inline size_t alloc_bytes(size_t bytes) { return ((bytes + 255) / 256) * 256 + 256; }

template <typename T>
fe_status dev_alloc(fe_ctx* c, T** p, size_t count) {
  size_t bytes = alloc_bytes(sizeof(T) * (count > 0 ? count : 1));
  cudaError_t e = cudaMalloc((void**)p, bytes);
  if (e != cudaSuccess) {
    *p = nullptr;
    return cuda_check(e, "cudaMalloc");
  }
  c->bytes += bytes;
  return FE_OK;
}

template <typename T>
void dev_free(fe_ctx* c, T** p, size_t count) {
  if (*p) {
    cudaFree(*p);
    size_t bytes = alloc_bytes(sizeof(T) * (count > 0 ? count : 1));
    c->bytes = c->bytes >= bytes ? c->bytes - bytes : 0;
  }
  *p = nullptr;
}

// Raise the dynamic shared-memory limit of kernel `func` to `bytes` on `device`, once per
// device (the attribute is per device); `done` is the caller's per-kernel bit mask of devices.
// Thread-safe: two threads may both set it, which is harmless.
inline fe_status ensure_smem(const void* func, int device, int bytes, std::atomic<uint64_t>& done) {
  const uint64_t bit = (device >= 0 && device < 64) ? (1ull << device) : 0ull;
  if (bit && (done.load(std::memory_order_acquire) & bit)) return FE_OK;
  const cudaError_t e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e != cudaSuccess) return cuda_check(e, "kernel shared-memory attribute");
  if (bit) done.fetch_or(bit, std::memory_order_release);
  return FE_OK;
}

// Number of SMs of `device`, queried once per device.
int sm_count(int device);

// fe_tiles.cu: the element tiles of the fused element + patch kernels (built from the
// device-order mesh; freed with the precompute).
fe_status build_tiles(fe_ctx* c);
void free_tiles(fe_ctx* c);

// fe_eval_f32.cu: bytes of one tile's FP32 element block, and the kernel that fills blk32 from
// dphi, vol and tile_elem (after the precompute).
size_t tile_block_bytes_f32(int dim);
fe_status launch_tile_blocks_f32(fe_ctx* c);

// Bracket a launch with profiling events when timing is enabled (no-op otherwise).
enum Stage { kStagePrep = 0, kStageElem = 1, kStageGather = 2, kStageFdElem = 3, kStageFdGather = 4 };
void prof_begin(fe_ctx* c, int stage);
void prof_end(fe_ctx* c, int stage);

}  // namespace fe
