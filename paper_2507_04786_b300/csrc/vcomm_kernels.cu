// vcomm_kernels.cu -- persistent collective kernels and their lookup table.
//
// One launch per collective call: grid = nranks x nsub CTAs, CTA b runs vrank
// b % nranks on channel (or tree sub-channel) b / nranks (Sec. V-D: one CUDA
// block per channel; here one block per (vrank, channel) because all vranks
// share the GPU).  All CTAs of a launch wait on one another through FIFO
// flags, so the host launches them cooperatively (co-residency guaranteed).
#include <cuda_runtime.h>

#include "vcomm_device.cuh"
#include "vcomm_kernels.h"

namespace vc {

template <int P>
__global__ void __launch_bounds__(maxThreadsFor(P), 1) kCopyColl(const __grid_constant__ KernArgs a) {
  __shared__ WorkerShared ws;
  if (threadIdx.x < 2) ws.abort[threadIdx.x] = 0;
  __syncthreads();
  const int r = blockIdx.x % a.nranks;
  const int ch = blockIdx.x / a.nranks;
  if (a.coll == kCopy) localCopy<uint8_t>(a, ch);
  else runWorker<P, uint8_t, OpNone>(a, r, ch, &ws);
}

// ---- protocol encoders exposed for tests: one thread per LL line pair / one
// warp per four LL128 lines, same device functions as the collectives
__global__ void kDebugEncode(int proto, const char* src, unsigned long long nbytes, uint64_t flag,
                             char* lines) {
  const unsigned long long gtid = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x;
  const unsigned long long gthr = (unsigned long long)gridDim.x * blockDim.x;
  if (proto == kLL) {
    const unsigned long long npairs = (nbytes + 7) / 8;
    for (unsigned long long p = gtid; p < npairs; p += gthr) {
      int valid = (int)((nbytes - 8 * p) < 8 ? (nbytes - 8 * p) : 8);
      llStorePair(lines, p, loadUser8<uint8_t>(src + 8 * p, valid), (uint32_t)flag);
    }
  } else {
    const unsigned long long nlines = (nbytes + 119) / 120;
    const unsigned long long nquads = (nlines + 3) / 4;
    const int lane = threadIdx.x & 31, j = lane & 7;
    for (unsigned long long q = gtid >> 5; q < nquads; q += gthr >> 5) {
      const unsigned long long line = 4 * q + (lane >> 3);
      if (line >= nlines) continue;
      const unsigned long long uoff = 120 * line + 16 * (unsigned long long)j;
      const int cap = (j == 7) ? 8 : 16;
      long long rem = (long long)nbytes - (long long)uoff;
      const int valid = rem <= 0 ? 0 : (rem < cap ? (int)rem : cap);
      uint64_t v0 = loadUser8<uint8_t>(src + uoff, valid < 8 ? valid : 8);
      uint64_t v1 = loadUser8<uint8_t>(src + uoff + 8, valid > 8 ? valid - 8 : 0);
      ll128Store(lines, line, j, v0, v1, flag);
    }
  }
}

__global__ void kDebugDecode(const __grid_constant__ KernArgs a, int proto, const char* lines,
                             unsigned long long nbytes, uint64_t flag, char* dst) {
  __shared__ int sAbort;
  if (threadIdx.x == 0) sAbort = 0;
  __syncthreads();
  volatile int* sa = &sAbort;
  const unsigned long long gtid = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x;
  const unsigned long long gthr = (unsigned long long)gridDim.x * blockDim.x;
  if (proto == kLL) {
    const unsigned long long npairs = (nbytes + 7) / 8;
    for (unsigned long long p = gtid; p < npairs; p += gthr) {
      int valid = (int)((nbytes - 8 * p) < 8 ? (nbytes - 8 * p) : 8);
      uint64_t v;
      if (!llLoadPair(a, lines, p, (uint32_t)flag, v, sa, 0, blockIdx.x)) return;
      storeUser8<uint8_t>(dst + 8 * p, v, valid);
    }
  } else {
    const unsigned long long nlines = (nbytes + 119) / 120;
    const unsigned long long nquads = (nlines + 3) / 4;
    const int lane = threadIdx.x & 31, j = lane & 7;
    for (unsigned long long q = gtid >> 5; q < nquads; q += gthr >> 5) {
      const unsigned long long line = 4 * q + (lane >> 3);
      const bool lineValid = line < nlines;
      const unsigned long long uoff = 120 * line + 16 * (unsigned long long)j;
      const int cap = (j == 7) ? 8 : 16;
      long long rem = lineValid ? (long long)nbytes - (long long)uoff : 0;
      const int valid = rem <= 0 ? 0 : (rem < cap ? (int)rem : cap);
      uint64_t v0, v1;
      if (!ll128Load(a, lines, line, lane, lineValid, flag, v0, v1, sa, 0, blockIdx.x)) return;
      storeUser8<uint8_t>(dst + uoff, v0, valid < 8 ? valid : 8);
      storeUser8<uint8_t>(dst + uoff + 8, v1, valid > 8 ? valid - 8 : 0);
    }
  }
}

// ---- lookup table
// reduce kernels are instantiated per (protocol, dtype) in vcomm_reduce_inst.cu
#define VC_DTYPES_OF(X, P) X(P, 0) X(P, 1) X(P, 2) X(P, 3) X(P, 4) X(P, 5) X(P, 6) X(P, 7) X(P, 8) X(P, 9)
#define VC_DECL(P, D) const void* reduceKernel_##P##_##D(int op);
VC_DTYPES_OF(VC_DECL, 0) VC_DTYPES_OF(VC_DECL, 1) VC_DTYPES_OF(VC_DECL, 2)
#undef VC_DECL

const void* reduceKernel(int proto, int dtype, int op) {
#define VC_CASE(P, D) if (proto == P && dtype == D) return reduceKernel_##P##_##D(op);
  VC_DTYPES_OF(VC_CASE, 0) VC_DTYPES_OF(VC_CASE, 1) VC_DTYPES_OF(VC_CASE, 2)
#undef VC_CASE
  return nullptr;
}

const void* copyKernel(int proto) {
  switch (proto) {
    case kSimple: return (const void*)kCopyColl<kSimple>;
    case kLL: return (const void*)kCopyColl<kLL>;
    case kLL128: return (const void*)kCopyColl<kLL128>;
  }
  return nullptr;
}

#define VC_CDECL(P, D) const void* clusterKernel_##D(int op);
VC_DTYPES_OF(VC_CDECL, 0)
#undef VC_CDECL
const void* clusterKernel(int dtype, int op) {
#define VC_CCASE(P, D) if (dtype == D) return clusterKernel_##D(op);
  VC_DTYPES_OF(VC_CCASE, 0)
#undef VC_CCASE
  return nullptr;
}

const void* debugEncodeKernel() { return (const void*)kDebugEncode; }
const void* debugDecodeKernel() { return (const void*)kDebugDecode; }

}  // namespace vc
