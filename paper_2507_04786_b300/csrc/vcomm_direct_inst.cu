// vcomm_direct_inst.cu -- the direct protocol's reducing kernels (single
// calls and grouped calls) for ONE dtype, selected by -DVC_DTYPE=<0..9>; the
// build compiles this file once per dtype.
#include <cuda_runtime.h>

#include "vcomm_direct.cuh"

#ifndef VC_DTYPE
#error "compile with -DVC_DTYPE=<0..9>"
#endif

namespace vc {
namespace direct {

template <class T, class Op>
__global__ void __launch_bounds__(DirectShape<T>::kThreads, 1)
    kDirectReduce(const __grid_constant__ DirectArgs a) {
  const DirectView v = viewOf(a);
  const bool last = blockIdx.x == gridDim.x - 1;
  unsigned long long lo, hi;
  if (a.vec == 1) {
    ctaRange(reduceUnits(v, Unit16<T>::kElems), &lo, &hi);
    directReduce<T, Op, Unit16<T>, DirectShape<T>::kUnits>(v, lo, hi, last);
  } else if (a.vec == 2) {
    ctaRange(shiftedUnits(v, (int)sizeof(T)), &lo, &hi);
    directReduceShifted<T, Op, PlainMem, DirectShape<T>::kUnits>(v, lo, hi, last);
  } else {
    ctaRange(reduceUnits(v, 1), &lo, &hi);
    directReduce<T, Op, Unit1<T>, 1>(v, lo, hi, last);
  }
}

template <class T, class Op>
__global__ void __launch_bounds__(DirectShape<T>::kThreads, 1)
    kDirectBatch(const __grid_constant__ DirectBatchArgs b) {
  const DirectBatchArgs* pb = &b;
  unsigned long long glo, ghi;
  ctaRange(pb->unitStart[pb->nops], &glo, &ghi);
  for (int i = 0; i < pb->nops; i++) {
    if (pb->unitStart[i + 1] <= glo || pb->unitStart[i] >= ghi) continue;
    unsigned long long lo, hi;
    bool tail;
    opShare(pb, i, glo, ghi, &lo, &hi, &tail);
    const DirectView v = viewOfOp(pb, i);
    // (2-byte types: one unit per thread, which the loop over ops leaves
    // registers for)
    constexpr int NU = sizeof(T) == 2 ? 1 : DirectShape<T>::kUnits;
    if (pb->ops[i].vec == 1) directReduce<T, Op, Unit16<T>, NU>(v, lo, hi, tail);
    else if (pb->ops[i].vec == 2) directReduceShifted<T, Op, PlainMem, 1>(v, lo, hi, tail);
    else directReduce<T, Op, Unit1<T>, 1>(v, lo, hi, tail);
  }
}

// AllReduce, ReduceScatter and Reduce of 16-byte aligned buffers staged
// through shared memory by bulk copies (one CTA per SM; dynamic shared memory
// from directStagedSmem)
template <class T, class Op>
__global__ void __launch_bounds__(256, 1) kDirectReduceStaged(const __grid_constant__ DirectArgs a) {
  directReduceStaged<T, Op>(a);
}

}  // namespace direct

using VcT = typename DTypeOf<VC_DTYPE>::T;

#define VC_DNAME2(N, D) N##_##D
#define VC_DNAME(N, D) VC_DNAME2(N, D)
const void* VC_DNAME(directReduceKernel, VC_DTYPE)(int op) {
  switch (op) {
    case kSum: case kAvg: return (const void*)direct::kDirectReduce<VcT, OpSum>;
    case kMax: return (const void*)direct::kDirectReduce<VcT, OpMax>;
    case kProd: return (const void*)direct::kDirectReduce<VcT, OpProd>;
    case kMin: return (const void*)direct::kDirectReduce<VcT, OpMin>;
  }
  return nullptr;
}
const void* VC_DNAME(directBatchKernel, VC_DTYPE)(int op) {
  switch (op) {
    case kSum: case kAvg: return (const void*)direct::kDirectBatch<VcT, OpSum>;
    case kMax: return (const void*)direct::kDirectBatch<VcT, OpMax>;
    case kProd: return (const void*)direct::kDirectBatch<VcT, OpProd>;
    case kMin: return (const void*)direct::kDirectBatch<VcT, OpMin>;
  }
  return nullptr;
}

}  // namespace vc

namespace vc {
const void* VC_DNAME(directStagedKernel, VC_DTYPE)(int op) {
  switch (op) {
    case kSum: case kAvg: return (const void*)direct::kDirectReduceStaged<VcT, OpSum>;
    case kMax: return (const void*)direct::kDirectReduceStaged<VcT, OpMax>;
    case kProd: return (const void*)direct::kDirectReduceStaged<VcT, OpProd>;
    case kMin: return (const void*)direct::kDirectReduceStaged<VcT, OpMin>;
  }
  return nullptr;
}
}  // namespace vc
