// Element epilogue shared by the CUDA-core and tensor-core GEMMs (semantics
// documented on GemmParams in ops.cuh).
#pragma once

#include "ops.cuh"

namespace kfm {

__device__ __forceinline__ double q_value(int q_kind, const double* q, int64_t ldq, int i, int j) {
  if (q_kind == 0) return i == j ? q[0] : 0.0;
  if (q_kind == 1) return i == j ? q[i] : 0.0;
  if (q_kind == 2) return q[(int64_t)i * ldq + j];
  return 0.0;
}

template <typename T>
__device__ __forceinline__ void epilogue_store(const GemmParams<T>& p, int gi, int gj, T acc) {
  T vpre = p.alpha * acc;
  if (p.cin) vpre += p.beta * p.cin[(int64_t)gi * p.ldcin + gj];
  T v = vpre;
  if (p.csub) v -= p.csub[(int64_t)gi * p.ldcsub + gj];
  const bool mirror = (p.sym == 1) && gi != gj;
  if (p.gain_q) {
    const T qi = (T)(p.gain_q_kind == 0 ? p.gain_q[0] : p.gain_q[gi]);
    const T qj = (T)(p.gain_q_kind == 0 ? p.gain_q[0] : p.gain_q[gj]);
    const T d = gi == gj ? T(1) : T(0);
    p.out[(int64_t)gi * p.ldo + gj] = d - qi * vpre;
    if (mirror) p.out[(int64_t)gj * p.ldo + gi] = d - qj * vpre;
    return;
  }
  if (p.out) {
    p.out[(int64_t)gi * p.ldo + gj] = v;
    if (mirror) p.out[(int64_t)gj * p.ldo + gi] = v;
  }
  if (p.outf) {
    p.outf[(int64_t)gi * p.ldof + gj] = (float)v;
    if (mirror) p.outf[(int64_t)gj * p.ldof + gi] = (float)v;
  }
  if (p.out2) {
    T w = vpre + (T)q_value(p.q_kind, p.q, p.ldq, gi, gj);
    p.out2[(int64_t)gi * p.ldo2 + gj] = w;
    if (mirror) p.out2[(int64_t)gj * p.ldo2 + gi] = w;
  }
  if (gi == gj) {
    if (p.diag_out) p.diag_out[gi] = (double)vpre;
    if (p.check_diag && !(vpre > T(0) && isfinite((double)vpre)))
      status_set(p.status, KF_ERR_NUMERIC, p.step, gi);
  }
}

}  // namespace kfm
