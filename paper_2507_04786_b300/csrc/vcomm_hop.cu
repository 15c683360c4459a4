// vcomm_hop.cu -- per-hop latency of the FIFO protocols (Sec. III: the
// protocols trade bandwidth for the latency of one hop; the paper quotes
// ~6 us Simple, ~1 us LL, ~2 us LL128 per hop on its hardware).
//
// A ring of n CTAs passes one FIFO line around `laps` times; CTA 0 times the
// laps with %globaltimer, so one hop = elapsed / (laps x n).  The ring's CTAs
// sit on chosen SMs: the kernel runs one CTA on every SM (a cooperative
// launch of nsm CTAs whose shared memory admits one per SM), each CTA reads
// its SM id and takes ring position pos[smid] (-1: not in the ring, return).
// Alternatively the ring is one thread-block cluster of n CTAs (cluster
// ranks 0..n-1), which the hardware places inside one GPC.
//
// One hop, per protocol:
//   LL    : the sender stores one 8-byte line {data, flag} (one st.volatile);
//           the receiver polls the line until its flag is the lap number.
//   LL128 : 8 lanes store the 128-byte line (the flag in its last 8 bytes)
//           with one warp-wide 16-byte store; 8 lanes of the receiver load it
//           and check the flag lane.
//   Simple: 8 lanes store a 128-byte payload, a gpu-scope fence, one release
//           store of the connection's counter; the receiver acquires the
//           counter, then loads the payload.
// Every wait is bounded by the timeout; a CTA that gives up records vTimeout
// and returns.
#include <cuda_runtime.h>

#include <vector>

#include "vcomm.h"
#include "vcomm_device.cuh"

namespace vc {
namespace {

// SM ids (%smid) need not be contiguous: the position table covers ids
// 0..kHopSmIds-1, and a CTA on an SM with a larger id takes no part
constexpr int kHopSmIds = 1024;

struct HopArgs {
  char* lines;                  // n incoming lines, 256 bytes apart (line i: into position i)
  const int* posOfSm;           // SM id -> ring position, -1 (SM-list mode); kHopSmIds entries
  int* smOfPos;                 // ring position -> SM id (written)
  unsigned long long* elapsed;  // written by position 0
  int* status;                  // vResult_t, first failure
  int n, laps, proto, cluster;
  unsigned long long timeoutNs;
};

VDEV int smid() {
  int s;
  asm volatile("mov.u32 %0, %%smid;" : "=r"(s));
  return s;
}

VDEV bool expired(const HopArgs& a, uint64_t t0) {
  if (globaltimer() - t0 > a.timeoutNs) {
    atomicCAS(a.status, 0, (int)vTimeout);
    return true;
  }
  return false;
}

// wait until the line into position `pos` carries lap `lap`; warp-collective
VDEV bool hopRecv(const HopArgs& a, int pos, uint64_t lap) {
  const int lane = threadIdx.x;
  char* line = a.lines + 256ull * pos;
  const uint64_t t0 = globaltimer();
  if (a.proto == kLL) {
    int ok = 0;
    if (lane == 0) {
      while (true) {
        uint64_t v = *(volatile uint64_t*)line;
        if ((uint32_t)(v >> 32) == (uint32_t)lap) { ok = 1; break; }
        if (*(volatile int*)a.status || expired(a, t0)) break;
      }
    }
    return __shfl_sync(0xffffffffu, ok, 0);
  }
  if (a.proto == kLL128) {
    uint64_t v0 = 0, v1 = 0;
    while (true) {
      if (lane < 8) ldVolatile2(line + 16 * lane, v0, v1);
      const bool mine = lane != 7 || v1 == lap;
      if (__all_sync(0xffffffffu, mine)) return true;
      int stop = 0;
      if (lane == 0) stop = *(volatile int*)a.status || expired(a, t0);
      if (__shfl_sync(0xffffffffu, stop, 0)) return false;
    }
  }
  // Simple: the counter, then the payload
  int ok = 0;
  unsigned long long* ctr = (unsigned long long*)(line + 128);
  if (lane == 0) {
    while (true) {
      if (ldAcquire(ctr) >= lap) { ok = 1; break; }
      if (*(volatile int*)a.status || expired(a, t0)) break;
    }
  }
  ok = __shfl_sync(0xffffffffu, ok, 0);
  if (ok && lane < 8) {
    const uint4 v = ldCG(line + 16 * lane);
    if (v.x == 0xffffffffu) atomicCAS(a.status, 0, (int)vInternalError);   // keeps the load
  }
  return ok;
}

VDEV void hopSend(const HopArgs& a, int pos, uint64_t lap) {
  const int lane = threadIdx.x;
  char* line = a.lines + 256ull * ((pos + 1) % a.n);
  if (a.proto == kLL) {
    if (lane == 0) *(volatile uint64_t*)line = (lap << 32) | (uint32_t)lap;
  } else if (a.proto == kLL128) {
    if (lane < 8) stVolatile2(line + 16 * lane, lap, lap);   // lane 7's second word is the flag
  } else {
    if (lane < 8) st16(line + 16 * lane, make_uint4((uint32_t)lap, 1, 2, 3));
    __threadfence();
    __syncwarp();
    if (lane == 0) stRelease((unsigned long long*)(line + 128), lap);
  }
}

__global__ void __launch_bounds__(32) kHopRing(const __grid_constant__ HopArgs a) {
  int pos;
  if (a.cluster) {
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    pos = (int)r;
  } else {
    const int id = smid();
    pos = (id >= 0 && id < kHopSmIds) ? a.posOfSm[id] : -1;
  }
  if (pos < 0 || pos >= a.n) return;
  if (threadIdx.x == 0) a.smOfPos[pos] = smid();
  uint64_t t0 = 0;
  for (uint64_t lap = 1; lap <= (uint64_t)a.laps; lap++) {
    if (pos == 0) {
      if (lap == 1) t0 = globaltimer();
      hopSend(a, pos, lap);
      if (!hopRecv(a, pos, lap)) return;
    } else {
      if (!hopRecv(a, pos, lap)) return;
      hopSend(a, pos, lap);
    }
  }
  if (pos == 0 && threadIdx.x == 0) *a.elapsed = globaltimer() - t0;
}

vResult_t fromCudaH(cudaError_t e) {
  if (e == cudaSuccess) return vSuccess;
  (void)cudaGetLastError();
  return e == cudaErrorMemoryAllocation ? vOutOfMemory : vCudaError;
}

}  // namespace
}  // namespace vc

using namespace vc;

extern "C" vResult_t vDebugHopLatency(vProto_t proto, const int* ringSms, int n, int laps, double timeoutSec,
                                      double* nsPerHop, int* smOut) {
  if (!nsPerHop || n < 2 || laps < 1 || timeoutSec <= 0) return vInvalidArgument;
  if (proto != vProtoSimple && proto != vProtoLL && proto != vProtoLL128) return vInvalidArgument;
  int dev = 0, nsm = 0;
  vResult_t r = fromCudaH(cudaGetDevice(&dev));
  if (r == vSuccess) r = fromCudaH(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  if (r != vSuccess) return r;
  const bool cluster = (ringSms == nullptr);
  if (cluster && n > 16) return vInvalidArgument;
  if (!cluster && n > nsm) return vInvalidArgument;
  std::vector<int> pos(kHopSmIds, -1);
  if (!cluster) {
    for (int i = 0; i < n; i++) {
      if (ringSms[i] < 0 || ringSms[i] >= kHopSmIds || pos[ringSms[i]] >= 0) return vInvalidArgument;
      pos[ringSms[i]] = i;
    }
  }
  char* lines = nullptr;
  int* dPos = nullptr;
  int* dSm = nullptr;
  unsigned long long* dEl = nullptr;
  int* dSt = nullptr;
  cudaStream_t s = nullptr;
  r = fromCudaH(cudaMalloc(&lines, 256ull * n));
  if (r == vSuccess) r = fromCudaH(cudaMemset(lines, 0, 256ull * n));
  if (r == vSuccess) r = fromCudaH(cudaMalloc(&dPos, sizeof(int) * kHopSmIds));
  if (r == vSuccess) r = fromCudaH(cudaMemcpy(dPos, pos.data(), sizeof(int) * kHopSmIds, cudaMemcpyHostToDevice));
  if (r == vSuccess) r = fromCudaH(cudaMalloc(&dSm, sizeof(int) * n));
  if (r == vSuccess) r = fromCudaH(cudaMemset(dSm, 0xff, sizeof(int) * n));
  if (r == vSuccess) r = fromCudaH(cudaMalloc(&dEl, sizeof(unsigned long long)));
  if (r == vSuccess) r = fromCudaH(cudaMemset(dEl, 0, sizeof(unsigned long long)));
  if (r == vSuccess) r = fromCudaH(cudaMalloc(&dSt, sizeof(int)));
  if (r == vSuccess) r = fromCudaH(cudaMemset(dSt, 0, sizeof(int)));
  if (r == vSuccess) r = fromCudaH(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
  HopArgs a;
  a.lines = lines;
  a.posOfSm = dPos;
  a.smOfPos = dSm;
  a.elapsed = dEl;
  a.status = dSt;
  a.n = n;
  a.laps = laps;
  a.proto = (int)proto - 1;
  a.cluster = cluster ? 1 : 0;
  a.timeoutNs = (unsigned long long)(timeoutSec * 1e9);
  if (r == vSuccess && cluster) {
    // one cluster of n CTAs (more than 8 needs the non-portable size)
    r = fromCudaH(cudaFuncSetAttribute(kHopRing, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = n;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(n);
    cfg.blockDim = dim3(32);
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (r == vSuccess) r = fromCudaH(cudaLaunchKernelEx(&cfg, kHopRing, a));
  } else if (r == vSuccess) {
    // one CTA per SM: shared memory that admits one CTA per SM, all CTAs
    // co-resident (cooperative launch), so every SM holds exactly one
    int maxSmem = 0;
    r = fromCudaH(cudaDeviceGetAttribute(&maxSmem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    const int smem = maxSmem;
    if (r == vSuccess)
      r = fromCudaH(cudaFuncSetAttribute(kHopRing, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    int per = 0;
    if (r == vSuccess) r = fromCudaH(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kHopRing, 32, smem));
    if (r == vSuccess && per != 1) r = vUnsupported;
    void* args[] = {(void*)&a};
    if (r == vSuccess)
      r = fromCudaH(cudaLaunchCooperativeKernel((const void*)kHopRing, dim3(nsm), dim3(32), args, smem, s));
  }
  if (r == vSuccess) r = fromCudaH(cudaStreamSynchronize(s));
  int st = 0;
  unsigned long long el = 0;
  if (r == vSuccess) r = fromCudaH(cudaMemcpy(&st, dSt, sizeof(int), cudaMemcpyDeviceToHost));
  if (r == vSuccess) r = fromCudaH(cudaMemcpy(&el, dEl, sizeof(el), cudaMemcpyDeviceToHost));
  if (r == vSuccess && smOut) r = fromCudaH(cudaMemcpy(smOut, dSm, sizeof(int) * n, cudaMemcpyDeviceToHost));
  if (r == vSuccess && st != 0) r = (vResult_t)st;
  if (r == vSuccess && el == 0) r = vTimeout;   // a ring SM id that no SM has: position 0 never ran
  if (r == vSuccess) *nsPerHop = (double)el / ((double)laps * n);
  if (lines) cudaFree(lines);
  if (dPos) cudaFree(dPos);
  if (dSm) cudaFree(dSm);
  if (dEl) cudaFree(dEl);
  if (dSt) cudaFree(dSt);
  if (s) cudaStreamDestroy(s);
  return r;
}
