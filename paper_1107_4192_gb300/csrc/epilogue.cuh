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
    if (p.outf) {
      p.outf[(int64_t)gi * p.ldof + gj] = (float)(d - qi * vpre);
      if (mirror) p.outf[(int64_t)gj * p.ldof + gi] = (float)(d - qj * vpre);
    }
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

// Row-pass / mirror-pass split of epilogue_store for kernels that stage a
// tile in shared memory (the tensor-core kernel): epilogue_row writes every
// direct output of element (gi, gj) and returns the value that its mirror
// (gj, gi) receives; epilogue_mirror writes the mirrored outputs from it
// (out2 with csub or a dense Q copies the direct element back, which the
// caller makes visible with a barrier between the two sweeps).
// cin_v / csub_v: the caller's preloaded cin[gi][gj] and csub[gi][gj] (zero when absent).
template <typename T>
__device__ __forceinline__ T epilogue_row(const GemmParams<T>& p, int gi, int gj, T acc, T cin_v, T csub_v) {
  T vpre = p.alpha * acc;
  if (p.cin) vpre += p.beta * cin_v;
  if (p.gain_q) {
    const T qi = (T)(p.gain_q_kind == 0 ? p.gain_q[0] : p.gain_q[gi]);
    const T jv = (gi == gj ? T(1) : T(0)) - qi * vpre;
    p.out[(int64_t)gi * p.ldo + gj] = jv;
    if (p.outf) p.outf[(int64_t)gi * p.ldof + gj] = (float)jv;
    return vpre;
  }
  T v = vpre;
  if (p.csub) v -= csub_v;
  if (p.out) p.out[(int64_t)gi * p.ldo + gj] = v;
  if (p.outf) p.outf[(int64_t)gi * p.ldof + gj] = (float)v;
  if (p.out2) p.out2[(int64_t)gi * p.ldo2 + gj] = vpre + (T)q_value(p.q_kind, p.q, p.ldq, gi, gj);
  if (gi == gj) {
    if (p.diag_out) p.diag_out[gi] = (double)vpre;
    if (p.check_diag && !(vpre > T(0) && isfinite((double)vpre)))
      status_set(p.status, KF_ERR_NUMERIC, p.step, gi);
  }
  return v;
}

// (gi, gj) is the mirrored position (gi < gj of the computed element's
// transpose); v is what epilogue_row returned for (gj, gi).
template <typename T>
__device__ __forceinline__ void epilogue_mirror(const GemmParams<T>& p, int gi, int gj, T v) {
  if (p.gain_q) {
    const T qi = (T)(p.gain_q_kind == 0 ? p.gain_q[0] : p.gain_q[gi]);
    p.out[(int64_t)gi * p.ldo + gj] = -qi * v;  // off-diagonal: delta = 0
    if (p.outf) p.outf[(int64_t)gi * p.ldof + gj] = (float)(-qi * v);
    return;
  }
  if (p.out) p.out[(int64_t)gi * p.ldo + gj] = v;
  if (p.outf) p.outf[(int64_t)gi * p.ldof + gj] = (float)v;
  if (p.out2) {
    // off the diagonal a diagonal Q adds nothing, so without csub the value is v;
    // otherwise copy the direct element (written in the row sweep) to stay bitwise symmetric
    const T w = (p.csub || p.q_kind == 2) ? p.out2[(int64_t)gj * p.ldo2 + gi] : v;
    p.out2[(int64_t)gi * p.ldo2 + gj] = w;
  }
}

}  // namespace kfm
