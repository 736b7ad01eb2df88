// On-chip sweep kernels (placeholder until the fast kernels land).
#include "qca_internal.cuh"

namespace qca {

int fast_path_for(int L, int v) {
  (void)L;
  (void)v;
  return 0;
}

int launch_fast(const DecodeArgs& a, cudaStream_t stream) {
  (void)a;
  (void)stream;
  set_error("no on-chip kernel for this size");
  return QCA_ERR_UNSUPPORTED;
}

}  // namespace qca
