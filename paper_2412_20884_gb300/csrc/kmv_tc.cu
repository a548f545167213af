// Tensor-core (tcgen05) forms of the kernel products.
#include "kmv_tc.cuh"

namespace kmv {

kmv_status tc_forward(kmv_handle h, const KmvArgs& a, cudaStream_t st) {
  (void)a; (void)st;
  h->last_error = "KMV_BF16_HILO is not built yet";
  return KMV_EUNSUPPORTED;
}

kmv_status tc_backward(kmv_handle h, const KmvArgs& a, double* grad, cudaStream_t st) {
  (void)a; (void)grad; (void)st;
  h->last_error = "KMV_BF16_HILO is not built yet";
  return KMV_EUNSUPPORTED;
}

void tc_release(kmv_handle h) { (void)h; }
size_t tc_workspace_bytes(kmv_handle h) { (void)h; return 0; }

}  // namespace kmv
