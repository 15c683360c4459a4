// vcomm_batch.cu -- the batched launch: many collectives, one persistent kernel.
//
// Group calls (Sec. II-A-4) defer a sequence of collectives so that they run
// as ONE launch.  The grid is a set of gangs; each gang is nranks x cpg CTAs
// and runs its ops one after another on its own channels, so ops of different
// gangs overlap on the device while ops of one gang pipeline through the same
// FIFOs.  CTA (r, ch) of a gang copies each op's description into shared
// memory (the paper's metadata-loading warp, Sec. V-D) and runs the op's
// (protocol, dtype, op) worker; CTAs whose channel the op does not use skip it.
#include <cuda_runtime.h>

#include "vcomm_device.cuh"
#include "vcomm_kernels.h"

namespace vc {

#define VC_DECL(P, D) __device__ void batchWorker_##P##_##D(const KernArgs&, int, int, volatile int*);
VC_DECL(0, 0) VC_DECL(0, 1) VC_DECL(0, 2) VC_DECL(0, 3)
VC_DECL(1, 0) VC_DECL(1, 1) VC_DECL(1, 2) VC_DECL(1, 3)
VC_DECL(2, 0) VC_DECL(2, 1) VC_DECL(2, 2) VC_DECL(2, 3)
#undef VC_DECL

template <int P>
__device__ __noinline__ void batchCopyWorker(const KernArgs& a, int r, int ch, volatile int* sAbort) {
  if (a.coll == kCopy) localCopy<uint8_t>(a, ch);
  else runWorker<P, uint8_t, OpNone>(a, r, ch, sAbort);
}

__device__ __forceinline__ void dispatchOp(const KernArgs& a, int proto, int dtype, bool bytes,
                                           int r, int ch, volatile int* sAbort) {
  if (bytes) {
    if (proto == kSimple) batchCopyWorker<kSimple>(a, r, ch, sAbort);
    else if (proto == kLL) batchCopyWorker<kLL>(a, r, ch, sAbort);
    else batchCopyWorker<kLL128>(a, r, ch, sAbort);
    return;
  }
#define VC_CASE(P, D) if (proto == P && dtype == D) { batchWorker_##P##_##D(a, r, ch, sAbort); return; }
  VC_CASE(0, 0) VC_CASE(0, 1) VC_CASE(0, 2) VC_CASE(0, 3)
  VC_CASE(1, 0) VC_CASE(1, 1) VC_CASE(1, 2) VC_CASE(1, 3)
  VC_CASE(2, 0) VC_CASE(2, 1) VC_CASE(2, 2) VC_CASE(2, 3)
#undef VC_CASE
}

__global__ void __launch_bounds__(512, 1) kBatch(const __grid_constant__ BatchArgs b) {
  __shared__ KernArgs sa;
  __shared__ int sAbort[2];
  const int k = b.nranks;
  const int per = k * b.cpg;
  const int gang = blockIdx.x / per;
  const int local = blockIdx.x % per;
  const int ch = local / k;
  const int r = local % k;
  if (threadIdx.x < 2) sAbort[threadIdx.x] = 0;
  for (int i = b.gangStart[gang]; i < b.gangStart[gang + 1]; i++) {
    const BatchOpDesc& o = b.ops[b.order[i]];
    if (ch >= o.nsub) continue;          // the op does not use this channel
    __syncthreads();                     // every thread is done with the previous op's sa
    if (threadIdx.x < k) {
      sa.send[threadIdx.x] = b.ptrs[o.ptrBase + threadIdx.x];
      sa.recv[threadIdx.x] = const_cast<void*>(b.ptrs[o.ptrBase + k + threadIdx.x]);
    }
    if (threadIdx.x == 0) {
      sa.count = o.count;
      sa.chunk = o.chunk;
      sa.slotBytes = o.slotBytes;
      sa.slotUnits = o.slotUnits;
      sa.timeoutNs = b.timeoutNs;
      sa.conns = o.conns ? const_cast<ConnDev*>(o.conns) + (unsigned long long)gang * b.cpg * k : nullptr;
      sa.errClaim = b.errClaim;
      sa.err = b.err;
      sa.abortFlag = b.abortFlag;
      sa.inplaceMask = o.inplaceMask;
      sa.downOffset = o.downOffset;
      sa.coll = o.coll;
      sa.algo = o.algo;
      sa.redop = o.redop;
      sa.nranks = k;
      sa.nsub = o.nsub;
      sa.root = o.root;
      sa.nsteps = b.nsteps;
      sa.upThreads = (blockDim.x / 2) / 32 * 32;
      sa.skipRank = -1;
    }
    __syncthreads();
    const bool bytes = (o.coll == kAllGather || o.coll == kBroadcast ||
                        (o.coll == kCopy && o.dtype < 0));
    dispatchOp(sa, o.proto, o.dtype, bytes, r, ch, sAbort);
    __syncthreads();
    if (sAbort[0] || sAbort[1]) return;  // a wait failed: the error word says where
  }
}

const void* batchKernel() { return (const void*)kBatch; }

}  // namespace vc
