// Host-side launchers of the device kernels.
#pragma once
#include <cuda_runtime.h>

#include <vector>

#include "hif_internal.h"

namespace hif {

// The largest shared memory a block may opt in to on the current device.
inline int smem_optin_max() {
  static const int v = [] {
    int dev = 0, x = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&x, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    return x > 0 ? x : 48 * 1024;
  }();
  return v;
}

// Raise kern's dynamic shared-memory limit to all the device allows next to
// the kernel's static shared memory (their sum may not exceed the opt-in
// maximum).  The value is fixed per kernel: host threads that launch the
// same kernel with different sizes (the batched API) must not set the limit
// to their own launch's size, or one would lower it under another's launch.
template <typename K>
inline void raise_smem_limit(K kern) {
  cudaFuncAttributes fa{};
  if (cudaFuncGetAttributes(&fa, kern) != cudaSuccess) return;
  const int lim = smem_optin_max() - (int)fa.sharedSizeBytes;
  if (lim > 0) cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
}


// factorization (kernels_factor.cu)
template <typename T>
// beta (host, dim values, NULL: none): a central-difference convection term
// beta . grad u, with F_IB stored for the cells that have room for it (FIB >= 0)
void launch_leaf_assemble(const CellDesc* cells, int ncells, const int* ipool, T* work, GridInfo g,
                          const double* a_stag, const double* bnode, const int* cls, int ncell_axis,
                          const double* beta, cudaStream_t st);
template <typename TU, typename TF>
void launch_extend_add(const CellDesc* cells, int ncells, const int* ipool, TF* work,
                       const CellDesc* pcells, const TU* pwork, int nchild, int max_nF, cudaStream_t st);
// sel (may be NULL: cells 0..ncells-1) lists the cells to factor; max_nI /
// max_nB over the listed cells
template <typename T>
void launch_cell_factor(const CellDesc* cells, const int* sel, int ncells, T* work, T* fac, int* status,
                        int max_nI, int max_nB, double tau, cudaStream_t st);
// tiled multi-block elimination of the problems td[0..n) (kernels_tiled.cu)
template <typename T>
void launch_tiled_elim(const TDesc* td, int n, int max_nI, int max_nB, T* work, T* fac, int* status, double tau,
                       cudaStream_t st, int tc_split = 0);
// tensor-core (tcgen05 TF32) panel solve + trailing update of panel p, and
// Schur complement, of the FP32 tiled elimination; return launches made
// (parts: TF32 parts per operand value, 1..3)
long long tc_panel(const TDesc* td, int nsel, int p, int P, int max_nI, int max_nB, float* work, int parts,
                   int* status, cudaStream_t st);
long long tc_syrk(const TDesc* td, int nsel, int max_nB, float* work, int parts, int* status, cudaStream_t st);
// U_b -= G_b G_b^T on nb contiguous blocks (G_b m x k, U_b m x m, row-major)
void tc_syrk_flat(int nb, int m, int k, const float* G, float* U, int parts, int* status, cudaStream_t st);
template <typename T>
void launch_front(const FrontDesc* fronts, int nfronts, const CellDesc* cells, const int* ipool, int* obuf,
                  T* fwork,
                  T* fac, T* cwork, double eps, int* status, int max_nc, int max_nN, double tau,
                  const int* sketch, SketchStream ss, const int* sel, cudaStream_t st);

// the two-sided (unsymmetric) factorization (kernels_twosided.cu): every
// cell of a level by LU (one block each, F_IB and the second factor set at
// the CellDesc's FIB / fac2), every front by the ID of [A_{N,c}; A_{c,N}^T]
// and the LU elimination of its redundant DOFs (FrontDesc fac2)
template <typename T>
void launch_cell_lu(const CellDesc* cells, const int* sel, int ncells, T* work, T* fac, int* status,
                    cudaStream_t st);
template <typename T>
void launch_front_lu(const FrontDesc* fronts, int nfronts, const CellDesc* cells, const int* ipool, int* obuf,
                     T* fwork, T* fac, T* cwork, double eps, int* status, int max_nc, int max_nN, cudaStream_t st);

// skeletonization by the SVD (kernels_svdfront.cu, Section 4.4): every front
// of a level (one block each), then the rotation of the update matrices of
// the cells ccell[0..ncells) by their fronts (cptr / clist: (front, side)
// pairs per cell, side 1 = P1, 2 = P2)
template <typename T>
void launch_front_svd(const FrontDesc* fronts, int nfronts, const CellDesc* cells, const int* ipool, int* obuf,
                      T* fwork, T* fac, const T* cwork, double eps, int* status, int max_nc, double tau,
                      cudaStream_t st);
template <typename T>
void launch_svd_rotate(const int* ccell, const int* cptr, const int* clist, int ncells, const FrontDesc* fronts,
                       const CellDesc* cells, const int* ipool, const int* obuf, const T* fwork, const T* fac,
                       T* cwork, int max_nc, cudaStream_t st);

// skeletonization of large fronts (kernels_bigfront.cu): the ID (writes T
// and the front's outputs; h_nc / h_nN: host copies of the fronts' sizes, for
// the block groups of the multi-block pivoted QR, used when coop_ok), then,
// with the ranks known on the host, the Lemma 2.4 blocks, and after the
// tiled elimination the B_ss scatter.
template <typename T>
void launch_bigfront_id(const FrontDesc* fronts, const int* big, int nbig, const CellDesc* cells, const int* ipool,
                        const T* cwork, T* fwork, T* fac, int* obuf, const int* sketch, SketchStream ss, double eps,
                        int* status, int* state, double* m2part, int nm, int max_nc,
                        int max_nN, int max_ell, const int* h_nc, const int* h_nN, bool coop_ok, cudaStream_t st);
template <typename T>
void launch_bigfront_form(const FrontDesc* fronts, const int* big, int nbig, const int* obuf, T* fwork,
                          const T* fac, int max_k, int max_nR, cudaStream_t st);
template <typename T>
void launch_bigfront_scatter(const FrontDesc* fronts, const int* big, int nbig, const CellDesc* cells,
                             const int* ipool, const int* obuf, const T* fwork, T* cwork, int max_k,
                             cudaStream_t st);
int bigfront_colmax_blocks(int max_nc);

// assembled upper levels of hifde3x (kernels_dense3x.cu): A is n_act x
// n_act, row-major; map[g] is the row of global DOF g (-1: not held)
template <typename TU, typename TA>
void launch_dense_from_cells(const CellDesc* cells, int ncells, const int* ipool, const TU* work, int max_nB,
                             const int* map, TA* A, int64_t n_act, cudaStream_t st);
// phase 0: gather F_II = A_pp, F_BI = A_qp, F_BB = 0; phase 1: A_qq += F_BB
template <typename T>
void launch_dense_cells(int phase, const CellDesc* cells, int ncells, const int* ipool, int max_nF,
                        const int* map, T* A, int64_t n_act, T* work, cudaStream_t st);
template <typename TA, typename TD>
void launch_dense_gather_root(const int* ids, int n, const int* map, const TA* A, int64_t n_act, TD* D,
                              cudaStream_t st);

// checks of the bounded device waits (each on an object nothing completes):
// the sweeps' bulk-copy wait (bit 3 of *err), the group barrier of the
// multi-block QR (bit 4), the tensor-core MMA wait (bit 5, with its TMEM freed)
void launch_wait_test_bulk(int* err, long polls, cudaStream_t st);
void launch_wait_test_group(unsigned* bar, int* err, long polls, cudaStream_t st);
void launch_wait_test_mma(int* status, uint64_t ns, cudaStream_t st);

// D^-1 of a root of at least kRootMulti DOFs by the whole GPU (kernels_root.cu):
// x_root <- L^-T S L^-1 x_root (S = diag(sgn)) on the rows ids[0..np) of x
// (N x nrhs, row stride ldx), in column chunks of kRootChunk; scratch:
// root_scratch_elems(np, det) elements (det: partial sums added in a fixed
// order instead of atomically).  Returns the number of launches.
constexpr int kRootMulti = 256;
constexpr int kRootChunk = 8;
int64_t root_scratch_elems(int np, bool det);
template <typename T>
int launch_root_apply(int np, const int* ids, const T* Linv, const T* sgn, T* x, int nrhs, int ldx, T* scratch,
                      bool det, cudaStream_t st);

// rank-prediction MLP (kernels_mlp.cu); idx may be NULL (samples 0..nb-1)
void mlp_grad(const float* X, const float* t, const int* idx, int nb, float inv_n, const float* prm,
              float* partial, float* ploss, float* grad, float* loss, cudaStream_t st);
void mlp_adam(float* prm, const float* grad, float* m, float* v, float lr, int t, cudaStream_t st);
void mlp_to_bf16(const float* prm, void* wbf16, cudaStream_t st);
void mlp_predict(const float* X, int n, const void* wbf16, float* y, cudaStream_t st);
int mlp_chunks(int nb);

// front features and sketch sizes (kernels_factor.cu)
void launch_front_features(const FrontDesc* fronts, int nfronts, const int* ipool, const double* stencil_w,
                           int dim, int n, int level, double eps, float* feats, cudaStream_t st);
void launch_sketch_sizes(const FrontDesc* fronts, int nfronts, const float* pred, int mode, int oversample,
                         int* sketch, cudaStream_t st);

// apply sweeps (kernels_apply.cu); op: 0 up, 1 down, 2 fwd_up, 3 fwd_down
// Launch shape of a sweep launch: threads per block (0: one per row and
// column group of the largest block, 32..256) and whether blocks stage their
// factor in shared memory (-1: when it fits, 0: never).
struct SweepShape {
  int threads = 0;
  int staged = -1;
};
// The deterministic scatter of one cell level: the ndof DOFs that the
// level's cells update (dofs[k]) with their contribution rows
// slots[ptr[k] .. ptr[k+1]) in cell order (row cslot + s of a cell is its
// s-th boundary DOF), and buf: one row of 32 elements of the apply's type per
// contribution.  With a plan, the cells' x_q updates of the F^-1 up sweep and
// the F fwd_down sweep are written to buf and summed per DOF by a second
// launch, so the result does not depend on the order the blocks run in.
struct ContribPlan {
  const int* ptr;
  const int* dofs;
  const int* slots;
  int ndof;
  void* buf;
};
template <typename T>
void launch_sweep(int op, const ApplyDesc* blocks, int nblocks, const int* ipool, const T* fac, T* x,
                  int nrhs, int ldx, int is_front, int max_np, int max_nq, int* err, cudaStream_t st,
                  SweepShape shape = SweepShape{}, const ContribPlan* cp = nullptr);

// F^-1 sweeps of the large blocks of a level by many thread blocks each
// (kernels_bigapply.cu): one BigBlock per block, scr = the offset of its
// scratch (2 np kBigChunk elements); dir 0 up, 1 down; max_np / max_nq over
// the blocks; scratch_elems: the level's scratch, zeroed here per chunk of
// kBigChunk right-hand sides.  Returns the launches made.
struct BigBlock {
  ApplyDesc d;
  int64_t scr;
};
constexpr int kBigChunk = 8;
template <typename T>
int launch_big_sweep(int dir, const BigBlock* bbs, int nbig, int max_np, int max_nq, int is_front, const int* ipool,
                     const T* fac, T* x, int nrhs, int ldx, T* scratch, int64_t scratch_elems, cudaStream_t st);

// stencil operator and CG vector operations (kernels_solve.cu)
void launch_matvec(GridInfo g, const double* a_stag, const double* b, const double* x, int ldx,
                   double* y, int ldy, int nr, cudaStream_t st);
void launch_mv_dot(GridInfo g, const double* a_stag, const double* b, const double* p, double* q,
                   int nr, double* partials, unsigned* counter, double* pq, cudaStream_t st);
void launch_axpy2(int64_t N, int nr, double* x, double* r, const double* p, const double* q,
                  const double* rz, const double* pq, const int* active, double* alpha,
                  double* partials, unsigned* counter, double* rr, cudaStream_t st);
void launch_dot2(int64_t N, int nr, const double* r, const double* z, const double* q,
                 double* partials, unsigned* counter, double* out, cudaStream_t st);
void launch_update_p(int64_t N, int nr, double* p, const double* z, const double* alpha,
                     const double* rz_old, const double* rzzq, const int* active, int restart,
                     cudaStream_t st);
void launch_residual(GridInfo g, const double* a_stag, const double* bn, const double* rhs,
                     const double* x, double* out, int nr, double* partials, unsigned* counter,
                     double* nrm2, cudaStream_t st);
void launch_sqnorm(int64_t N, int nr, const double* v, double* partials, unsigned* counter,
                   double* out, cudaStream_t st);
void launch_dd_residual(GridInfo g, const double* a_stag, const double* bn, const double* f,
                        const double* xh, const double* xl, double* r, int nr, double* partials,
                        unsigned* counter, double* nrm2, cudaStream_t st);
void launch_dd_add(int64_t N, int nr, double* xh, double* xl, const double* d, cudaStream_t st);
// element-parallel CG kernels on N x R vectors, R in {1, 2, 4, 8, 16}
void launch_stencil_weights(GridInfo g, const double* a_stag, const double* b, double* W, cudaStream_t st);
// q = A p, pq = p.q; with alpha (may be NULL): alpha = rz / pq on the active columns
void launch_mv_dot_e(GridInfo g, const double* W, const double* p, double* q, int R, double* partials,
                     unsigned* counter, double* pq, cudaStream_t st, const double* rz = nullptr,
                     const int* active = nullptr, double* alpha = nullptr);
template <typename TZ>
void launch_axpy2_e(int64_t N, int R, double* x, double* r, const double* p, const double* q,
                    const double* alpha, double* partials, unsigned* counter, double* rr, TZ* zin, cudaStream_t st,
                    const double* thr2 = nullptr, int* active_next = nullptr, double* ring_rr = nullptr);
// out = [r.z | z.q]; beta = -alpha zq / rz_old
template <typename TZ>
void launch_dot2_e(int64_t N, int R, const double* r, const TZ* z, const double* q, double* partials,
                   unsigned* counter, double* out, cudaStream_t st, double* ring_rz, const double* alpha,
                   const double* rz_old, double* beta);
template <typename TZ>
void launch_update_p_e(int64_t N, int R, double* p, const TZ* z, const double* beta, const double* rz_old,
                       const int* active, int restart, cudaStream_t st);
void launch_set_active(int nr, const double* rr, const double* thr2, int* active, cudaStream_t st);
// flexible GMRES: basis slabs V_i = V + i slab (N x R); out[i R + c] = <V_i, w>
void launch_multi_dot(int64_t N, int R, const double* V, int64_t slab, int nv, const double* w, double* partials,
                      unsigned* counters, double* out, cudaStream_t st);
void launch_multi_axpy(int64_t N, int R, const double* V, int64_t slab, int nv, const double* h, double* w,
                       cudaStream_t st);
void launch_normalize(int64_t N, int R, const double* w, const double* nrm2, double* v, double* hnorm,
                      cudaStream_t st);
template <typename TZ>
void launch_zy_add(int64_t N, int R, const TZ* Z, int64_t slab, int nv, const double* y, double* d,
                   cudaStream_t st);
template <typename TI, typename TO>
void launch_convert(int64_t N, int nr, const TI* in, int ldi, TO* out, int ldo, cudaStream_t st);

}  // namespace hif
