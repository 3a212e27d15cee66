// tcgen05 / TMA Gram passes of a run group: one launch per pass over the
// runs that share the form, kernel kind and distance tile (k_group_tc in
// kkm_gram_tc.cuh). A translation unit of its own so that it compiles beside
// the single-run one.
#include "kkm_gram_tc.cuh"

namespace kkm {
namespace {

template <int KIND, int MODE, int OP, int TNV>
cudaError_t launch_group_form(const GroupPhase& g, int ctas, cudaStream_t st) {
  static std::atomic<uint64_t> attr{0};
  {
    const cudaError_t e = smem_limit_once(k_group_tc<KIND, MODE, OP, TNV>, smem_bytes<TNV>(), attr);
    if (e != cudaSuccess) return e;
  }
  return launch_pdl(k_group_tc<KIND, MODE, OP, TNV>, dim3(ctas), dim3(NTHREADS), smem_bytes<TNV>(), st, g);
}

template <int MODE, int OP, int TNV>
cudaError_t launch_group_kind(const GroupPhase& g, int kind, int ctas, cudaStream_t st) {
  switch (kind) {
    case K_GAUSS: return launch_group_form<K_GAUSS, MODE, OP, TNV>(g, ctas, st);
    case K_LAPLACE: return launch_group_form<K_LAPLACE, MODE, OP, TNV>(g, ctas, st);
    case K_LINEAR: return launch_group_form<K_LINEAR, MODE, OP, TNV>(g, ctas, st);
    default: return launch_group_form<K_POLY, MODE, OP, TNV>(g, ctas, st);
  }
}

template <int MODE, int TNV>
cudaError_t launch_group_op(const GroupPhase& g, int form, int kind, int ctas, cudaStream_t st) {
  switch (form) {
    case FORM_BF16X3: return launch_group_kind<MODE, OP_X3, TNV>(g, kind, ctas, st);
    case FORM_TF32: return launch_group_kind<MODE, OP_TF32, TNV>(g, kind, ctas, st);
    default: return launch_group_kind<MODE, OP_BF16, TNV>(g, kind, ctas, st);
  }
}

}  // namespace

cudaError_t launch_group_tc(const GroupPhase& g, int mode, int form, int kind, int tn, int ctas, cudaStream_t st) {
  if (ctas <= 0) return cudaSuccess;
  if (mode == 1) return launch_group_op<1, WPASS_TNV>(g, form, kind, ctas, st);
  if (tn == 64) return launch_group_op<0, 64>(g, form, kind, ctas, st);
  if (tn == 256) return launch_group_op<0, 256>(g, form, kind, ctas, st);
  return launch_group_op<0, 128>(g, form, kind, ctas, st);
}

}  // namespace kkm
