// Placeholder until the tcgen05 kernel lands: reports the path as unavailable.
#include "tc_gemm.cuh"

namespace kfm {

uint64_t tc_scratch_bytes(int64_t rows, int64_t ld) { return 4ull * rows * ld * sizeof(__nv_bfloat16); }

kf_status tc_scratch_alloc(TcScratch& sc, int64_t rows, int64_t ld,
                           const std::function<kf_status(void**, size_t)>& alloc) {
  size_t plane = (size_t)rows * ld * sizeof(__nv_bfloat16);
  KF_TRY(alloc((void**)&sc.a_hi, plane));
  KF_TRY(alloc((void**)&sc.a_lo, plane));
  KF_TRY(alloc((void**)&sc.b_hi, plane));
  KF_TRY(alloc((void**)&sc.b_lo, plane));
  sc.rows = rows;
  sc.ld = ld;
  return KF_OK;
}

bool tc_available() { return false; }

kf_status tc_gemm_bf16x3(cudaStream_t, TcScratch&, const GemmParams<float>&) { return KF_ERR_UNSUPPORTED; }

}  // namespace kfm
