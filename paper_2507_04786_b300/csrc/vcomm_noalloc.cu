// vcomm_noalloc.cu -- vAllReduceNoAlloc: a ring AllReduce that allocates nothing.
//
// For callers that must not allocate device memory at call time: code that
// runs under a fixed memory budget owned by another allocator, code on a
// latency-critical path where cudaMalloc / cudaFree could block or implicitly
// synchronise the device, and embedders that have no communicator object to
// keep.  Instead of a communicator's FIFO arena, the connections live in one
// file-scope device array of fixed size, which every GPU that loads this
// library holds until the process exits.  The paper has no counterpart; the
// kernel itself is the ordinary Simple-protocol ring AllReduce.
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>
#include <mutex>

#include "vcomm.h"
#include "vcomm_internal.h"
#include "vcomm_kernels.h"

using namespace vc;

namespace {

constexpr int kNaSlots = 4;                                     // FIFO slots per connection
constexpr size_t kNaSlotBytes = 64u << 10;                      // one slot: 64 KiB
constexpr size_t kNaFifoBytes = (size_t)VCOMM_NOALLOC_MAX_CONNS * kNaSlots * kNaSlotBytes;
constexpr size_t kNaCtrBytes = (size_t)VCOMM_NOALLOC_MAX_CONNS * 2 * kCounterStride * 8;
constexpr size_t kNaConnBytes = (size_t)VCOMM_NOALLOC_MAX_CONNS * sizeof(ConnDev);
constexpr size_t kNaCtrOff = kNaFifoBytes;
constexpr size_t kNaConnOff = kNaCtrOff + kNaCtrBytes;
constexpr size_t kNaErrOff = kNaConnOff + kNaConnBytes;         // ErrWord, claim word, abort word
constexpr size_t kNaTotal = kNaErrOff + 256;
static_assert(kNaTotal == VCOMM_NOALLOC_SCRATCH_BYTES, "scratch size in vcomm.h is stale");

}  // namespace

// The scratch itself.  In host code this name is only a host-side stand-in:
// the device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char gNoAllocScratch[kNaTotal];

namespace {

// The device address of gNoAllocScratch, looked up once per device ordinal and
// kept for the life of the process.  cudaDeviceReset destroys the context
// that holds it (the module is loaded again, maybe elsewhere), so calls must
// not span a reset of the device.
constexpr int kNaMaxDevices = 64;
std::mutex gNaMu;
void* gNaBase[kNaMaxDevices];

// every call clears what must start at zero (counters, error words) and
// rebuilds the connection table: the previous call's contents are stale
__global__ void kNoAllocSetup(unsigned char* base, int nconn, int* status) {
  unsigned long long* ctr = (unsigned long long*)(base + kNaCtrOff);
  ConnDev* conns = (ConnDev*)(base + kNaConnOff);
  for (int i = threadIdx.x; i < VCOMM_NOALLOC_MAX_CONNS * 2 * kCounterStride; i += blockDim.x) ctr[i] = 0;
  for (int i = threadIdx.x; i < nconn; i += blockDim.x) {
    conns[i].buf = (char*)base + (size_t)i * kNaSlots * kNaSlotBytes;
    conns[i].tail = ctr + (size_t)(2 * i) * kCounterStride;
    conns[i].head = ctr + (size_t)(2 * i + 1) * kCounterStride;
    conns[i].unused = 0;
  }
  if (threadIdx.x < 64) ((int*)(base + kNaErrOff))[threadIdx.x] = 0;
  if (status && threadIdx.x < 4) status[threadIdx.x] = 0;
}

bool overlap(uintptr_t a, uintptr_t b, size_t n) { return a < b + n && b < a + n; }

}  // namespace

extern "C" vResult_t vAllReduceNoAlloc(const void* const* sendbufs, void* const* recvbufs,
                                       size_t count, vDataType_t dtype, vRedOp_t op, int nranks,
                                       int nchannels, int* deviceStatus, vStream_t stream) {
  if (!sendbufs || !recvbufs) return vInvalidArgument;
  if (nranks < 1 || nranks > VCOMM_MAX_RANKS || nchannels < 1) return vInvalidArgument;
  if ((long long)nranks * nchannels > VCOMM_NOALLOC_MAX_CONNS) return vInvalidArgument;
  if (dtype < vInt32 || dtype > vBfloat16 || op < vSum || op > vMax) return vInvalidArgument;
  if (count == 0) return vSuccess;
  const size_t esz = (dtype == vFloat16 || dtype == vBfloat16) ? 2 : 4;
  const size_t nb = count * esz;
  unsigned long long inplace = 0;
  for (int r = 0; r < nranks; r++) {
    uintptr_t s = (uintptr_t)sendbufs[r], d = (uintptr_t)recvbufs[r];
    if (!s || !d || s % esz || d % esz) return vInvalidArgument;
    if (s == d) inplace |= 1ull << r;
    else if (overlap(s, d, nb)) return vInvalidArgument;
    for (int q = 0; q < r; q++) {
      if (overlap(d, (uintptr_t)recvbufs[q], nb) || overlap(d, (uintptr_t)sendbufs[q], nb) ||
          overlap((uintptr_t)recvbufs[q], s, nb))
        return vInvalidArgument;
    }
  }

  // set-up, once per device, with that device current: the scratch's address
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    (void)cudaGetLastError();
    return vCudaError;
  }
  if (dev < 0 || dev >= kNaMaxDevices) return vUnsupported;
  unsigned char* base = nullptr;
  {
    std::lock_guard<std::mutex> lk(gNaMu);
    if (!gNaBase[dev]) {
      void* p = nullptr;
      cudaError_t e = cudaGetSymbolAddress(&p, gNoAllocScratch);
      if (e != cudaSuccess || !p) {
        (void)cudaGetLastError();
        return vCudaError;
      }
      gNaBase[dev] = p;
    }
    base = (unsigned char*)gNaBase[dev];
  }

  const int k = nranks;
  const int kcoll = (k == 1) ? kCopy : kAllReduce;
  KernArgs a;
  memset(&a, 0, sizeof(a));
  for (int r = 0; r < k; r++) {
    a.send[r] = sendbufs[r];
    a.recv[r] = recvbufs[r];
  }
  a.count = count;
  a.slotBytes = kNaSlotBytes;
  a.slotUnits = kNaSlotBytes / esz;
  a.chunk = kNaSlotBytes / esz;               // chunkCount = one slot of data
  a.timeoutNs = 5000000000ull;
  a.conns = (ConnDev*)(base + kNaConnOff);
  a.err = deviceStatus ? (ErrWord*)deviceStatus : (ErrWord*)(base + kNaErrOff);
  a.errClaim = (int*)(base + kNaErrOff + 64);
  a.abortFlag = (const volatile int*)(base + kNaErrOff + 128);
  a.inplaceMask = inplace;
  a.downOffset = 0;
  a.coll = kcoll;
  a.algo = kRing;
  a.nranks = k;
  a.nsub = nchannels;
  a.root = 0;
  a.nsteps = kNaSlots;
  a.upThreads = 0;
  a.skipRank = -1;

  cudaStream_t s = (cudaStream_t)stream;
  kNoAllocSetup<<<1, 256, 0, s>>>(base, k * nchannels, deviceStatus);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return vCudaError;
  const void* fn = reduceKernel(kSimple, dtype, op);
  if (!fn) return vInternalError;
  // k x C <= 32 CTAs of 256 threads are always co-resident on a B300
  void* args[] = {(void*)&a};
  e = cudaLaunchCooperativeKernel(fn, dim3((unsigned)(k * nchannels)), dim3(256), args, 0, s);
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    return vCudaError;
  }
  return vSuccess;
}
