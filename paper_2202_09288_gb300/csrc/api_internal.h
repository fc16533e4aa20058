// api_internal.h -- internal hooks of api.cu used by other translation units of the
// library.  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "../../include/chol.h"

namespace chol {

size_t solve_scratch_doubles(const chol_num* f, int64_t k);
int enqueue_solve_ws(chol_ctx* c, const chol_num* f, int k, const double* B, int64_t ldb,
                     double* X, int64_t ldx, double* ws);
int check_solve_args(chol_ctx* c, const chol_num* f, int64_t nrhs, const double* B,
                     int64_t ldb, const double* X, int64_t ldx, int64_t* n_out);
cudaStream_t ctx_stream(const chol_ctx* c);
int ctx_device(const chol_ctx* c);

}  // namespace chol
