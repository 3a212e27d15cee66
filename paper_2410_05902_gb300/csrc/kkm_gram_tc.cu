// tcgen05 / TMA Gram passes of one run: the tensor maps, the launch
// configuration and the entry points of kkm_internal.cuh. The kernels are in
// kkm_gram_tc.cuh.
#include "kkm_gram_tc.cuh"

namespace kkm {
namespace {

template <int KIND, int MODE, int OP, int TNV>
cudaError_t launch_form(const Dev& s, const CUtensorMap& a, const CUtensorMap& b, int rows, cudaStream_t st) {
  static std::atomic<uint64_t> attr{0};
  {
    const cudaError_t e = smem_limit_once(k_dist_tc<KIND, MODE, OP, TNV>, smem_bytes<TNV>(), attr);
    if (e != cudaSuccess) return e;
  }
  // one CTA per SM, but never more CTAs than the most items this launch can
  // have: small runs then leave SMs free for the kernels of other runs
  const int64_t most = MODE == 0 ? (int64_t)((rows + TM - 1) / TM) * s.max_tiles : (int64_t)s.max_pairs;
  const int grid = (int)(most < s.num_sms ? (most > 0 ? most : 1) : s.num_sms);
  return launch_pdl(k_dist_tc<KIND, MODE, OP, TNV>, dim3(grid), dim3(NTHREADS), smem_bytes<TNV>(), st, s, rows, a,
                    b);
}

template <int MODE, int OP, int TNV>
cudaError_t launch_kind(const Dev& s, const CUtensorMap& a, const CUtensorMap& b, int rows, cudaStream_t st) {
  switch (s.kind) {
    case K_GAUSS: return launch_form<K_GAUSS, MODE, OP, TNV>(s, a, b, rows, st);
    case K_LAPLACE: return launch_form<K_LAPLACE, MODE, OP, TNV>(s, a, b, rows, st);
    case K_LINEAR: return launch_form<K_LINEAR, MODE, OP, TNV>(s, a, b, rows, st);
    default: return launch_form<K_POLY, MODE, OP, TNV>(s, a, b, rows, st);
  }
}

// maps: [0] batch rows, 128-row boxes; support rows with [1] 128-row, [2] 64-row, [3] 256-row boxes
template <int MODE, int TNV>
cudaError_t launch_mode(const Dev& s, const void* maps_in, int rows, cudaStream_t st) {
  const CUtensorMap* m = static_cast<const CUtensorMap*>(maps_in);
  const CUtensorMap& a = (MODE == 0) ? m[0] : m[1];
  const CUtensorMap& b = (TNV == 256) ? m[3] : (TNV == 128) ? m[1] : m[2];
  switch (s.form) {
    case FORM_BF16X3: return launch_kind<MODE, OP_X3, TNV>(s, a, b, rows, st);
    case FORM_TF32: return launch_kind<MODE, OP_TF32, TNV>(s, a, b, rows, st);
    default: return launch_kind<MODE, OP_BF16, TNV>(s, a, b, rows, st);
  }
}

// The passes' failure-detection path: thread 0 waits on an mbarrier of one
// arrival with the passes' bounded wait. With arrive = 0 nothing arrives, so
// the wait runs out after limit_ns; out[0] = 1 if it did.
__global__ void k_wait_probe(uint64_t limit_ns, int arrive, int* out) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x != 0) return;
  mbar_init(&bar, 1);
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  if (arrive) mbar_arrive(&bar);
  out[0] = mbar_wait(&bar, 0, limit_ns) ? 0 : 1;
  mbar_inval(&bar);
}

}  // namespace

cudaError_t launch_wait_probe(uint64_t limit_ns, int arrive, int* out, cudaStream_t st) {
  k_wait_probe<<<1, 32, 0, st>>>(limit_ns, arrive, out);
  return cudaGetLastError();
}

// Tensor maps of the batch rows and the support store: 2-D tensors of ld
// columns (BF16, or FP32 for the TF32 form), boxes of one 128-byte row of
// columns (64 BF16 or 32 FP32) x 128 (64, 256) rows, 128-byte swizzle.
cudaError_t tc_prepare(Dev& s, void* maps_out) {
  static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  if (!encode) {
    cudaDriverEntryPointQueryResult q;
    void* fn = nullptr;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                                     cudaEnableDefault, &q);
    if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn) return cudaErrorNotSupported;
    encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  }
  CUtensorMap* maps = static_cast<CUtensorMap*>(maps_out);
  const int64_t srows = (int64_t)s.k * s.cap + 256;
  const bool f32 = s.form == FORM_TF32;
  void* xb = f32 ? (void*)s.xb32 : (void*)s.xbh;
  void* yb = f32 ? (void*)s.y32 : (void*)s.ybh;
  const int esz = f32 ? 4 : 2;
  struct { void* base; uint64_t rows; uint32_t box_rows; } ops[4] = {
      {xb, (uint64_t)s.bpad, 128u}, {yb, (uint64_t)srows, 128u}, {yb, (uint64_t)srows, 64u},
      {yb, (uint64_t)srows, 256u}};
  for (int i = 0; i < 4; ++i) {
    cuuint64_t dims[2] = {(cuuint64_t)s.ld, (cuuint64_t)ops[i].rows};
    cuuint64_t strides[1] = {(cuuint64_t)s.ld * esz};
    cuuint32_t box[2] = {(cuuint32_t)(128 / esz), ops[i].box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = encode(&maps[i], f32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2,
                        ops[i].base, dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
  }
  return cudaSuccess;
}

int tc_parts_per_tile(int tn) {
  return tn == 256 ? Geo<256>::GPT : tn == 64 ? Geo<64>::GPT : Geo<128>::GPT;
}

cudaError_t launch_dist_tc(const Dev& s, const void* maps, int rows, cudaStream_t st, bool stage_early) {
  if (rows <= 0) return cudaSuccess;
  // staging before the grid-dependency wait is only safe when the kernel just
  // ahead writes none of what it stages (the gather, or this pass itself)
  Dev d = s;
  d.pre_b = (stage_early && s.pre_b) ? 1 : 0;
  if (d.tn == 64) return launch_mode<0, 64>(d, maps, rows, st);
  if (d.tn == 256) return launch_mode<0, 256>(d, maps, rows, st);
  return launch_mode<0, 128>(d, maps, rows, st);
}

cudaError_t launch_wgram_tc(const Dev& s, const void* maps, cudaStream_t st) {
  return launch_mode<1, WPASS_TNV>(s, maps, 0, st);
}

}  // namespace kkm
