// kernels.h -- host-callable launchers of the device kernels (factor_kernels.cu,
// solve_kernels.cu).  All launches are asynchronous on the given stream.
#pragma once

#include <cuda_runtime.h>

#include "chol_internal.h"

namespace chol {

void launch_assemble(const double* vals, const int64_t* amap, int64_t nnz, void* L, bool f32,
                     cudaStream_t st);
// Task launches run one CTA per task (launch_util.h); a grid smaller than the task list would
// take further tasks from the zero-initialized work-queue counter `queue` (one per launch).
// Widest supernode whose diagonal-block inverse the factor keeps (for the solves).
constexpr int kDinvMaxWidth = 64;
// Y = L11^-1 of every supernode of a POTRF task list whose descriptor has dinv set (the
// blocks are final: after launch_potrf of the same level); with skip_sliced, not those whose
// task has its y field set (FP64 POTRF formed their Y already).
void launch_diag_inverse(const int4* tasks, int ntasks, const SnDev* sns, bool f32,
                         bool skip_sliced, cudaStream_t st);
// oy: with the FP64 factor's tensor-core TRSM, the zeroed scratch (oz_scratch_bytes(oy_rows))
// that receives the slices of the 128-tile supernodes' Y = L11^-1 (tasks with y set); else null
void launch_potrf(const int4* tasks, int ntasks, int* queue, const SnDev* sns,
                  const MatDev* mats, int max_width, bool f32, float tau, void* oy,
                  int64_t oy_rows, cudaStream_t st);
void launch_trsm(const int4* tasks, int ntasks, int* queue, const SnDev* sns, int max_width,
                 bool f32, cudaStream_t st);
void launch_schur(int cls, const int4* tasks, int ntasks, int* queue, const SnDev* sns,
                  const MatDev* mats, bool owner, bool f32, cudaStream_t st);
void launch_assemble_owner(const int4* groups, int ngroups, int* queue, const int4* srcs,
                           const SnDev* sns, const MatDev* mats, bool f32, cudaStream_t st);
int set_factor_kernel_attrs(int max_width);
// The relative map of a pattern (MatDev::relmap), one CTA per supernode; misses counted.
void launch_build_relmap(int32_t ns, const int32_t* sn_start, const int64_t* sn_rowptr,
                         const int32_t* rows, const int32_t* sn_run0, const int32_t* run_a,
                         const int32_t* run_t, const int64_t* run_base, int32_t* relmap,
                         unsigned long long* miss, cudaStream_t st);
// 128 x 128 FP32 Schur tiles on the tcgen05 tensor cores (3xTF32), tc_kernels.cu: per
// level, the hi/lo TF32 parts of the 128-tile supernodes' L21 (kTaskOzSlice tasks) into the
// zeroed scratch oz (oz_scratch_bytes(oz_rows)), then the tiles.
void launch_tf32_split(const int4* tasks, int ntasks, const SnDev* sns, int max_width, void* oz,
                       int64_t oz_rows, cudaStream_t st);
// acc_wait: 0 normally; > 0 is a test hook of the failure path: the consumer warps then wait
// acc_wait SM clock cycles on a barrier that never completes (an accumulator that never
// finishes) and give up.
void launch_schur_tc(const int4* tasks, int ntasks, int* queue, const SnDev* sns,
                     const MatDev* mats, bool owner, const void* oz, int64_t oz_rows,
                     long long acc_wait, cudaStream_t st);
int set_tc_kernel_attrs();
// FP64 128 x 128 Schur tiles on the bf16 tensor cores by operand splitting, oz_kernels.cu:
// per level, first the slices of every 128-tile supernode's L21 (kTaskOzSlice tasks), then
// the tiles.  oz is a zeroed scratch of oz_scratch_bytes(oz_rows) bytes.
// oy: null for the Schur tiles' L21; for the tensor-core TRSM's A21, the inverses' scratch
// (the columns are scaled by the shifts POTRF stored there)
void launch_oz_slice(const int4* tasks, int ntasks, const SnDev* sns, void* oz, int64_t oz_rows,
                     const void* oy, int64_t oy_rows, cudaStream_t st);
void launch_schur_oz(const int4* tasks, int ntasks, int* queue, const SnDev* sns,
                     const MatDev* mats, bool owner, const void* oz, int64_t oz_rows,
                     long long acc_wait, cudaStream_t st);
// L21 = A21 Y^T of the 128-tile supernodes on the bf16 tensor cores (kTaskOzSlice tasks: 128
// rows each): A21's slices from launch_oz_slice with oy on the panel before this launch, Y's
// slices from launch_potrf (oy); writes L21 into the panels.
void launch_trsm_oz(const int4* tasks, int ntasks, const SnDev* sns, const MatDev* mats,
                    const void* oz, int64_t oz_rows, const void* oy, int64_t oy_rows,
                    cudaStream_t st);
size_t oz_scratch_bytes(int64_t oz_rows);
// the inverses' slice scratch: slice planes, row exponents, then one column shift per row
size_t oy_scratch_bytes(int64_t oy_rows);
int set_oz_kernel_attrs();

void launch_gather_perm(const double* B, int64_t ldb, const int32_t* perm, const double* scale,
                        int64_t n, int nrhs, double* y, cudaStream_t st);
void launch_scatter_perm(const double* w, const int32_t* perm, const double* scale, int64_t n,
                         int nrhs, double* X, int64_t ldx, cudaStream_t st);
// W: the level's widest supernode (launch sizes); inv: the factor keeps the inverses of its
// diagonal blocks
void launch_fwd(const int4* tasks, int ntasks, int* queue, const SnDev* sns, int64_t ldv,
                int nrhs, int W, double* y, double* w, double* fstage, bool inv, bool f32,
                cudaStream_t st);
void launch_fwd_gather(const int32_t* fg_row, const int64_t* fg_ptr, const int32_t* fg_ent,
                       int64_t nrows, int64_t ldv, int nrhs, const double* fstage, double* y,
                       cudaStream_t st);
// queue: the level's work-queue counter; arrive: one zeroed counter per supernode (the
// backward step's last-task detection); W: the stride of the partial slots (the width cap);
// wl: the level's widest supernode (launch sizes)
void launch_bwd(const int4* tasks, int ntasks, int* queue, const SnDev* sns, int64_t ldv,
                int nrhs, int W, int wl, double* w, double* part, int* arrive, bool inv,
                bool f32, cudaStream_t st);
int set_solve_kernel_attrs(int W, int max_nrhs);

void launch_diag_scale(const int64_t* colptr, const int32_t* rowind, const double* vals,
                       const int32_t* iperm, int64_t n, double* scale, unsigned long long* err,
                       cudaStream_t st);
void launch_assemble_scaled(const int64_t* colptr, const int32_t* rowind, const double* vals,
                            const int64_t* amap, const double* scale, int64_t n, float* L,
                            cudaStream_t st);
void launch_residual(const int64_t* ptr, const int32_t* col, const int32_t* src,
                     const double* vals, int64_t n, int nrhs, const double* X, int64_t ldx,
                     const double* B, int64_t ldb, double* R, int64_t ldr, cudaStream_t st);
void launch_absmax(const double* V, int64_t ld, int64_t n, int nrhs, unsigned long long* out,
                   cudaStream_t st);
void launch_anorm(const int64_t* ptr, const int32_t* src, const double* vals, int64_t n,
                  unsigned long long* out, cudaStream_t st);
void launch_axpy(double* X, int64_t ldx, const double* D, int64_t ldd, int64_t n, int nrhs,
                 cudaStream_t st);

}  // namespace chol
