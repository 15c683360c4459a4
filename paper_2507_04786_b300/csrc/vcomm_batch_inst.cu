// vcomm_batch_inst.cu -- the batch kernel's worker for ONE (protocol, dtype)
// pair, selected by -DVC_PROTO / -DVC_DTYPE (compiled once per pair, as
// relocatable device code, and called from vcomm_batch.cu).
#include <cuda_runtime.h>

#include "vcomm_device.cuh"

#ifndef VC_PROTO
#error "compile with -DVC_PROTO=<0|1|2> -DVC_DTYPE=<0..9>"
#endif

namespace vc {

using VcT = typename DTypeOf<VC_DTYPE>::T;

#define VC_BNAME2(P, D) batchWorker_##P##_##D
#define VC_BNAME(P, D) VC_BNAME2(P, D)

// one reduction op's worker, not inlined so that each gets its own register
// allocation (templated on the protocol and type too: this unit is linked as
// relocatable device code with its siblings, so the name must be unique)
template <int P, class T, class Op>
__device__ __noinline__ void opWorker(const KernArgs& a, int r, int ch, WorkerShared* ws) {
  runWorker<P, T, Op>(a, r, ch, ws);
}

// one op of a batch on CTA (r, ch) of its gang; `a` lives in shared memory
__device__ __noinline__ void VC_BNAME(VC_PROTO, VC_DTYPE)(const KernArgs& a, int r, int ch,
                                                         WorkerShared* ws) {
  if (a.coll == kCopy) localCopy<VcT>(a, ch);
  else if (a.redop == kSum) opWorker<VC_PROTO, VcT, OpSum>(a, r, ch, ws);
  else if (a.redop == kMax) opWorker<VC_PROTO, VcT, OpMax>(a, r, ch, ws);
  else if (a.redop == kProd) opWorker<VC_PROTO, VcT, OpProd>(a, r, ch, ws);
  else if (a.redop == kMin) opWorker<VC_PROTO, VcT, OpMin>(a, r, ch, ws);
  else opWorker<VC_PROTO, VcT, OpAvg>(a, r, ch, ws);
}

}  // namespace vc
