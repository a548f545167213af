// Tensor-core (tcgen05) forms of the kernel products; see kmv_tc.cu.
#pragma once

#include "kmv_internal.cuh"

namespace kmv {

// Y = A(theta) V with the KMV_BF16_HILO arithmetic.  Honours a.sys_active,
// a.col_shift, a.Y64 and a.dot_partial like the SIMT form.
kmv_status tc_forward(kmv_handle h, const KmvArgs& a, cudaStream_t st);
// Adjoint with the KMV_BF16_HILO arithmetic; writes grad (systems, n_theta)
// and, when a.Y != NULL, dL/dV = A G into a.Y.
kmv_status tc_backward(kmv_handle h, const KmvArgs& a, double* grad, cudaStream_t st);
// True when a one- or two-column KMV_BF16_HILO product takes the FMA-pipe
// path with the three-way exponent split (relative operator error ~1e-6).
bool x_width_fma_ok(int d);
// Frees the tensor-core path's own workspace.
void tc_release(kmv_handle h);
size_t tc_workspace_bytes(kmv_handle h);

}  // namespace kmv
