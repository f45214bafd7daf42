// fe_cg.cu -- Steihaug's truncated conjugate gradients (Nocedal & Wright, Alg. 7.2) for the
// trust-region subproblem  min_z g.z + z.H z / 2,  ||z|| <= radius,  with H the Hessian of the
// discrete energy at v (the products of fe_hessian.cu).  Not in the paper, whose trust-region
// solver is a closed toolbox; this is the inner solver of a trust-region Newton method driven
// by the kernels.
//
// Everything runs on the device.  The solver's scalars live in a CgState in device memory;
// every kernel reads them at entry, so all blocks take the same branch, and the block that
// finishes a kernel's reduction last (a ticket counter) writes the new scalars and the flags.
// One CG iteration is five launches on the context stream:
//   k_w_prep + k_hvp_cached_f64 + k_gather_bulk   Hd = H d (the v-dependent terms of H are
//                                           computed once per solve by k_hvp_prep_f64)
//   k_cg_curv                               dHd = d.Hd
//   k_cg_step                               z += a d, Hz += a Hd, r += a Hd; r.r, z.z
//                                           (a = r.r / dHd, or the step to the boundary)
//   k_cg_dir                                d = -r + beta d; d.d, z.d
// The host enqueues iterations in batches (2, 4, ... 32) and reads the state between batches;
// launches enqueued after the solve has finished see the done flag and return at once.
// The dot products are the fixed-order reductions of reduce.cuh, so results are bitwise
// reproducible.
#include "fe_internal.cuh"
#include "reduce.cuh"

namespace fe {
namespace {

// tau >= 0 with ||z + tau d|| = radius, from zz = z.z, zd = z.d, dd = d.d.
__device__ __forceinline__ double cg_to_boundary(double zz, double zd, double dd, double radius2) {
  const double disc = fmax(fma(zd, zd, dd * (radius2 - zz)), 0.0);
  return (sqrt(disc) - zd) / fmax(dd, 1e-300);
}

__global__ void __launch_bounds__(kThreads) k_cg_init(int64_t n, const double* __restrict__ g, double* __restrict__ z,
                                                      double* __restrict__ Hz, double* __restrict__ r,
                                                      double* __restrict__ d, CgState* st, double* part,
                                                      unsigned* ticket, double radius, double tol, int max_cg) {
  double acc[1] = {0.0};
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const double gi = g[i];
    z[i] = 0.0;
    Hz[i] = 0.0;
    r[i] = gi;
    d[i] = -gi;
    acc[0] = fma(gi, gi, acc[0]);
  }
  double tot[1];
  if (red_finish<1>(acc, part, ticket, tot)) {
    st->rr = st->rrn = st->dd = tot[0];
    st->zd = st->zz = st->dHd = 0.0;
    st->radius2 = radius * radius;
    st->tol = tol;
    st->k = 0;
    st->max_cg = max_cg;
    st->boundary = 0;
    st->done = (sqrt(tot[0]) <= tol || max_cg <= 0) ? 1 : 0;
  }
}

__global__ void __launch_bounds__(kThreads) k_cg_curv(int64_t n, const double* __restrict__ d,
                                                      const double* __restrict__ Hd, CgState* st, double* part,
                                                      unsigned* ticket) {
  if (st->done) return;
  double acc[1] = {0.0};
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
    acc[0] = fma(d[i], Hd[i], acc[0]);
  double tot[1];
  if (red_finish<1>(acc, part, ticket, tot)) st->dHd = tot[0];
}

__global__ void __launch_bounds__(kThreads) k_cg_step(int64_t n, double* __restrict__ z, double* __restrict__ Hz,
                                                      double* __restrict__ r, const double* __restrict__ d,
                                                      const double* __restrict__ Hd, CgState* st, double* part,
                                                      unsigned* ticket) {
  if (st->done) return;
  const double dHd = st->dHd, rr = st->rr, zz = st->zz, zd = st->zd, dd = st->dd, R2 = st->radius2;
  // non-positive curvature, or a step that leaves the ball: move to the boundary and stop
  bool stop = !(dHd > 0.0);
  double a = stop ? 0.0 : rr / dHd;
  if (!stop && fma(a * a, dd, fma(2.0 * a, zd, zz)) >= R2) stop = true;
  if (stop) a = cg_to_boundary(zz, zd, dd, R2);
  double acc[2] = {0.0, 0.0};
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const double di = d[i], hi = Hd[i];
    const double zi = fma(a, di, z[i]);
    z[i] = zi;
    Hz[i] = fma(a, hi, Hz[i]);
    if (!stop) {
      const double ri = fma(a, hi, r[i]);
      r[i] = ri;
      acc[0] = fma(ri, ri, acc[0]);
      acc[1] = fma(zi, zi, acc[1]);
    }
  }
  double tot[2];
  if (red_finish<2>(acc, part, ticket, tot)) {
    const int k = st->k + 1;
    st->k = k;
    if (stop) {
      st->boundary = 1;
      st->done = 1;
    } else {
      st->rrn = tot[0];
      st->zz = tot[1];
      if (sqrt(tot[0]) <= st->tol || k >= st->max_cg) st->done = 1;
    }
  }
}

__global__ void __launch_bounds__(kThreads) k_cg_dir(int64_t n, const double* __restrict__ z,
                                                     const double* __restrict__ r, double* __restrict__ d,
                                                     CgState* st, double* part, unsigned* ticket) {
  if (st->done) return;
  const double beta = st->rrn / st->rr;
  double acc[2] = {0.0, 0.0};
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const double di = fma(beta, d[i], -r[i]);
    d[i] = di;
    acc[0] = fma(di, di, acc[0]);
    acc[1] = fma(z[i], di, acc[1]);
  }
  double tot[2];
  if (red_finish<2>(acc, part, ticket, tot)) {
    st->dd = tot[0];
    st->zd = tot[1];
    st->rr = st->rrn;
  }
}

}  // namespace

fe_status launch_cg_steihaug(fe_ctx* c, const double* v, const double* g, double radius, double tol, int max_cg,
                             double* z, double* Hz, int* iters, int* boundary) {
  cudaStream_t s = c->stream;
  const int64_t n = c->nn * c->d;
  double* r = c->cg_vec;
  double* d = r + n;
  double* Hd = d + n;
  CgState* st_dev = c->cg_state;
  const int* skip = &st_dev->done;
  const int nb = grid_for(n, kMaxNodeBlocks);
  fe_status st = launch_hvp_prepare_f64(c, v);
  if (st) return st;
  k_cg_init<<<nb, kThreads, 0, s>>>(n, g, z, Hz, r, d, st_dev, c->cg_part, c->cg_ticket, radius, tol, max_cg);
  c->launches++;
  if ((st = cuda_check(cudaGetLastError(), "cg init"))) return st;
  // Each non-skipped step raises k by one and sets done at k == max_cg, so the solve ends
  // within max_cg iterations; the bound below only guards the host loop.
  const int64_t limit = (int64_t)(max_cg > 0 ? max_cg : 0) + 64;
  int64_t issued = 0;
  int batch = 2;
  for (;;) {
    for (int b = 0; b < batch; ++b) {
      if ((st = launch_hvp_cached_f64(c, d, Hd, skip))) return st;
      k_cg_curv<<<nb, kThreads, 0, s>>>(n, d, Hd, st_dev, c->cg_part, c->cg_ticket);
      k_cg_step<<<nb, kThreads, 0, s>>>(n, z, Hz, r, d, Hd, st_dev, c->cg_part, c->cg_ticket);
      k_cg_dir<<<nb, kThreads, 0, s>>>(n, z, r, d, st_dev, c->cg_part, c->cg_ticket);
      c->launches += 3;
    }
    issued += batch;
    if ((st = cuda_check(cudaMemcpyAsync(c->cg_host, st_dev, sizeof(CgState), cudaMemcpyDeviceToHost, s),
                         "cg state read")))
      return st;
    if ((st = cuda_check(cudaStreamSynchronize(s), "cg sync"))) return st;
    if (c->cg_host->done) break;
    if (issued > limit) return set_error(FE_ECUDA, "conjugate gradients did not finish");
    batch = batch < 32 ? 2 * batch : 32;
  }
  *iters = c->cg_host->k;
  *boundary = c->cg_host->boundary;
  return FE_OK;
}

}  // namespace fe
