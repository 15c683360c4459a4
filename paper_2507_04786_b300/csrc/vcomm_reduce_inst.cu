// vcomm_reduce_inst.cu -- the reducing collective kernel for ONE (protocol,
// dtype) pair, selected at compile time by -DVC_PROTO=<0..2> -DVC_DTYPE=<0..9>.
// The build compiles this file once per pair, in parallel.
#include <cuda_runtime.h>

#include "vcomm_device.cuh"

#ifndef VC_PROTO
#error "compile with -DVC_PROTO=<0|1|2> -DVC_DTYPE=<0..9>"
#endif

namespace vc {

template <int P, class T, class Op>
__global__ void __launch_bounds__(maxThreadsFor(P), 1) kReduceColl(const __grid_constant__ KernArgs a) {
  __shared__ WorkerShared ws;
  if (threadIdx.x < 2) ws.abort[threadIdx.x] = 0;
  __syncthreads();
  const int r = blockIdx.x % a.nranks;
  const int ch = blockIdx.x / a.nranks;
  if (a.coll == kCopy) localCopy<T>(a, ch);
  else runWorker<P, T, Op>(a, r, ch, &ws);
}

using VcT = typename DTypeOf<VC_DTYPE>::T;

#define VC_NAME2(P, D) reduceKernel_##P##_##D
#define VC_NAME(P, D) VC_NAME2(P, D)
const void* VC_NAME(VC_PROTO, VC_DTYPE)(int op) {
  switch (op) {
    case kSum: return (const void*)kReduceColl<VC_PROTO, VcT, OpSum>;
    case kMax: return (const void*)kReduceColl<VC_PROTO, VcT, OpMax>;
    case kProd: return (const void*)kReduceColl<VC_PROTO, VcT, OpProd>;
    case kMin: return (const void*)kReduceColl<VC_PROTO, VcT, OpMin>;
    case kAvg: return (const void*)kReduceColl<VC_PROTO, VcT, OpAvg>;
  }
  return nullptr;
}

}  // namespace vc
