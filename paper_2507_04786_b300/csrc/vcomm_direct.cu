// vcomm_direct.cu -- the direct protocol: collectives with no FIFO.
//
// Sec. IV describes P2P_DIRECT: ranks of one process move data straight
// between source and destination buffers (directSend / directRecv) instead of
// through an intermediate FIFO.  With every vrank in one GPU's memory this
// goes one step further: a thread reads the k input buffers of one 16-byte
// unit itself and folds them in exactly the order the ring schedule would
// (Table "Ring AllReduce": segment s starts at rank s + 1 and ends at rank s;
// ReduceScatter block b likewise from rank b + 1; Reduce from root + 1), so
// the partial sums of the chain never leave registers.  Each input byte is
// read once and each output byte written once: 2kS bytes for a k-vrank
// AllReduce of S bytes per vrank, against 2kS + 4(k-1)S for the Simple ring.
// The segments come from the same partition (channels, loops, chunkCount) as
// the FIFO kernels, so for a given plan the results are the Simple
// protocol's, bit for bit.
//
// No thread waits for another: a plain launch of a grid sized to the data.
#include <cuda_runtime.h>

#include "vcomm_direct.cuh"
#include "vcomm_kernels.h"

namespace vc {
namespace direct {

__global__ void __launch_bounds__(256) kDirectCopy(const __grid_constant__ DirectArgs a) {
  const DirectView v = viewOf(a);
  const bool last = blockIdx.x == gridDim.x - 1;
  unsigned long long lo, hi;
  if (a.vec == 1) {
    ctaRange(copyUnits(v, 16), &lo, &hi);
    directCopy<Unit16<uint8_t>>(v, lo, hi, last);
  } else if (a.vec == 2) {
    ctaRange(shiftedUnits(v, 1), &lo, &hi);
    directCopyShifted<PlainMem>(v, lo, hi, last);
  } else {
    ctaRange(copyUnits(v, 1), &lo, &hi);
    directCopy<Unit1<uint8_t>>(v, lo, hi, last);
  }
}

__global__ void __launch_bounds__(256) kDirectBatchCopy(const __grid_constant__ DirectBatchArgs b) {
  const DirectBatchArgs* pb = &b;
  unsigned long long glo, ghi;
  ctaRange(pb->unitStart[pb->nops], &glo, &ghi);
  for (int i = 0; i < pb->nops; i++) {
    if (pb->unitStart[i + 1] <= glo || pb->unitStart[i] >= ghi) continue;
    unsigned long long lo, hi;
    bool tail;
    opShare(pb, i, glo, ghi, &lo, &hi, &tail);
    const DirectView v = viewOfOp(pb, i);
    if (pb->ops[i].vec == 1) directCopy<Unit16<uint8_t>>(v, lo, hi, tail);
    else if (pb->ops[i].vec == 2) directCopyShifted<PlainMem>(v, lo, hi, tail);
    else directCopy<Unit1<uint8_t>>(v, lo, hi, tail);
  }
}

// AllGather, Broadcast and point-to-point transfers of 16-byte aligned
// buffers staged through shared memory by bulk copies; one thread of the
// CTA drives them
__global__ void __launch_bounds__(32) kCopyStaged(const __grid_constant__ CopyArgs a) { copyStaged(a); }

}  // namespace direct

#define VC_DDECL(D) const void* directReduceKernel_##D(int op); const void* directBatchKernel_##D(int op); \
  const void* directStagedKernel_##D(int op);
VC_DDECL(0) VC_DDECL(1) VC_DDECL(2) VC_DDECL(3) VC_DDECL(4)
VC_DDECL(5) VC_DDECL(6) VC_DDECL(7) VC_DDECL(8) VC_DDECL(9)
#undef VC_DDECL

static int dtypeBytes(int dtype) {
  switch (dtype) {
    case kI8: case kU8: return 1;
    case kF16: case kBF16: return 2;
    case kI64: case kU64: case kF64: return 8;
  }
  return 4;
}

int directThreads(int coll, int dtype) {
  if (coll == kAllGather || coll == kBroadcast) return 256;
  return direct::directThreadsFor(dtypeBytes(dtype));
}

const void* directKernel(int coll, int dtype, int op) {
  if (coll == kAllGather || coll == kBroadcast) return (const void*)direct::kDirectCopy;
  switch (dtype) {
#define VC_DCASE(D) case D: return directReduceKernel_##D(op);
    VC_DCASE(0) VC_DCASE(1) VC_DCASE(2) VC_DCASE(3) VC_DCASE(4)
    VC_DCASE(5) VC_DCASE(6) VC_DCASE(7) VC_DCASE(8) VC_DCASE(9)
#undef VC_DCASE
  }
  return nullptr;
}

const void* directBatchKernel(int coll, int dtype, int op) {
  if (coll == kAllGather || coll == kBroadcast) return (const void*)direct::kDirectBatchCopy;
  switch (dtype) {
#define VC_DCASE(D) case D: return directBatchKernel_##D(op);
    VC_DCASE(0) VC_DCASE(1) VC_DCASE(2) VC_DCASE(3) VC_DCASE(4)
    VC_DCASE(5) VC_DCASE(6) VC_DCASE(7) VC_DCASE(8) VC_DCASE(9)
#undef VC_DCASE
  }
  return nullptr;
}

const void* directStagedKernel(int dtype, int op) {
  switch (dtype) {
#define VC_DCASE(D) case D: return directStagedKernel_##D(op);
    VC_DCASE(0) VC_DCASE(1) VC_DCASE(2) VC_DCASE(3) VC_DCASE(4)
    VC_DCASE(5) VC_DCASE(6) VC_DCASE(7) VC_DCASE(8) VC_DCASE(9)
#undef VC_DCASE
  }
  return nullptr;
}

int directStagedThreads() { return 256; }

int directStagedMaxStages() { return direct::kMaxStages; }

const void* copyStagedKernel() { return (const void*)direct::kCopyStaged; }
int copyStagedMaxStages() { return direct::kMaxCopyStages; }

size_t directStagedSmem(int nranks, int stages, unsigned tileBytes) {
  return (size_t)stages * nranks * tileBytes + 2 * (size_t)tileBytes + 8 * (size_t)stages;
}

unsigned directStagedTile(int nranks, int stages, size_t smemMax) {
  const size_t per = (size_t)stages * nranks + 2;   // tiles held in shared memory
  const size_t t = (smemMax - 8 * (size_t)stages) / per / 128 * 128;
  return (unsigned)(t < 128 ? 128 : t > 16384 ? 16384 : t);
}

}  // namespace vc
