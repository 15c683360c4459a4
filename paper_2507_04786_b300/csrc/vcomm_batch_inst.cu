// vcomm_batch_inst.cu -- the batch kernel's worker for ONE (protocol, dtype)
// pair, selected by -DVC_PROTO / -DVC_DTYPE (compiled once per pair, as
// relocatable device code, and called from vcomm_batch.cu).
#include <cuda_runtime.h>

#include "vcomm_device.cuh"

#ifndef VC_PROTO
#error "compile with -DVC_PROTO=<0|1|2> -DVC_DTYPE=<0..3>"
#endif

namespace vc {

#if VC_DTYPE == 0
using VcT = int32_t;
#elif VC_DTYPE == 1
using VcT = float;
#elif VC_DTYPE == 2
using VcT = __half;
#else
using VcT = __nv_bfloat16;
#endif

#define VC_BNAME2(P, D) batchWorker_##P##_##D
#define VC_BNAME(P, D) VC_BNAME2(P, D)

// one op of a batch on CTA (r, ch) of its gang; `a` lives in shared memory
__device__ __noinline__ void VC_BNAME(VC_PROTO, VC_DTYPE)(const KernArgs& a, int r, int ch,
                                                         volatile int* sAbort) {
  if (a.coll == kCopy) localCopy<VcT>(a, ch);
  else if (a.redop == kSum) runWorker<VC_PROTO, VcT, OpSum>(a, r, ch, sAbort);
  else runWorker<VC_PROTO, VcT, OpMax>(a, r, ch, sAbort);
}

}  // namespace vc
