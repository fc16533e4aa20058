// kernels.h -- host-callable launchers of the device kernels (factor_kernels.cu,
// solve_kernels.cu).  All launches are asynchronous on the given stream.
#pragma once

#include <cuda_runtime.h>

#include "chol_internal.h"

namespace chol {

void launch_assemble(const double* vals, const int64_t* amap, int64_t nnz, void* L, bool f32,
                     cudaStream_t st);
void launch_potrf(const int4* tasks, int ntasks, const SnDev* sns, const MatDev* mats,
                  int max_width, cudaStream_t st);
void launch_trsm(const int4* tasks, int ntasks, const SnDev* sns, int max_width,
                 cudaStream_t st);
void launch_schur(int cls, const int4* tasks, int ntasks, const SnDev* sns, const MatDev* mats,
                  double* stage, bool owner, cudaStream_t st);
void launch_assemble_owner(const int4* groups, int ngroups, const int4* srcs, const SnDev* sns,
                           const MatDev* mats, const double* stage, cudaStream_t st);
int set_factor_kernel_attrs(int max_width);

void launch_gather_perm(const double* B, int64_t ldb, const int32_t* perm, int64_t n, int nrhs,
                        double* y, cudaStream_t st);
void launch_scatter_perm(const double* w, const int32_t* perm, int64_t n, int nrhs, double* X,
                         int64_t ldx, cudaStream_t st);
void launch_fwd(const int4* tasks, int ntasks, const SnDev* sns, int64_t ldv, int nrhs, int W,
                double* y, double* w, double* fstage, cudaStream_t st);
void launch_fwd_gather(const int32_t* fg_row, const int64_t* fg_ptr, const int32_t* fg_ent,
                       int64_t nrows, int64_t ldv, int nrhs, const double* fstage, double* y,
                       cudaStream_t st);
void launch_bwd(const int4* bwd_tasks, int nbwd, int64_t bwd_base, const int4* diag_tasks,
                int ndiag, const SnDev* sns, int64_t ldv, int nrhs, int W, double* w,
                double* part, cudaStream_t st);
int set_solve_kernel_attrs(int W, int max_nrhs);

}  // namespace chol
