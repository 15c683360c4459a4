// vcomm_cluster_inst.cu -- cluster-protocol kernels for ONE dtype, selected by
// -DVC_DTYPE=<0..9> (compiled once per dtype); the dtype-0 unit also holds
// the byte-moving kernel for AllGather and Broadcast.
#include <cuda_runtime.h>

#include "vcomm_cluster.cuh"

#ifndef VC_DTYPE
#error "compile with -DVC_DTYPE=<0..9>"
#endif

namespace vc {

using VcT = typename DTypeOf<VC_DTYPE>::T;

// one cluster of nranks CTAs per channel (launched with that cluster shape)
template <class T, class Op>
__global__ void __launch_bounds__(maxThreadsFor(kCluster), 1) kClusterColl(const __grid_constant__ KernArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int sAbort[2];
  if (threadIdx.x < 2) sAbort[threadIdx.x] = 0;
  __syncthreads();
  if (a.nranks == 1) {   // single rank: a copy of the channel's range
    localCopy<T>(a, blockIdx.x);
    return;
  }
  const int r = blockIdx.x % a.nranks;
  const int ch = blockIdx.x / a.nranks;
  runClusterWorker<T, Op>(a, r, ch, sAbort, smem);
}

#define VC_CNAME2(D) clusterKernel_##D
#define VC_CNAME(D) VC_CNAME2(D)
const void* VC_CNAME(VC_DTYPE)(int op) {
  switch (op) {
    case kSum: return (const void*)kClusterColl<VcT, OpSum>;
    case kMax: return (const void*)kClusterColl<VcT, OpMax>;
    case kProd: return (const void*)kClusterColl<VcT, OpProd>;
    case kMin: return (const void*)kClusterColl<VcT, OpMin>;
    case kAvg: return (const void*)kClusterColl<VcT, OpAvg>;
  }
  return nullptr;
}

#if VC_DTYPE == 0
const void* clusterCopyKernel() { return (const void*)kClusterColl<uint8_t, OpNone>; }
#endif

}  // namespace vc
