// vcomm_host.cu -- host runtime behind include/vcomm.h.
//
// The communicator (Sec. II-A-1, ncclCommInitAll) owns one FIFO arena per
// (algorithm, protocol), the host-mapped error and abort words, and the plan
// state.  Each collective call validates its arguments, picks a plan
// (algorithm, protocol, channels, chunk steps: Sec. II-C and III-D), and
// enqueues ONE cooperative launch of the persistent kernel on the caller's
// stream.  Nothing here touches user data.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <utility>
#include <vector>

#include "vcomm.h"
#include "vcomm_internal.h"
#include "vcomm_kernels.h"

using namespace vc;

namespace {

struct Arena {
  bool ready = false;
  ConnDev* dConns = nullptr;
  char* dBuf = nullptr;
  unsigned long long* dCtr = nullptr;
  int nconn = 0;
  size_t bytes = 0;
};

constexpr size_t kDefaultSlot[3] = {512u << 10, 32u << 10, 600u << 10};

vResult_t fromCuda(cudaError_t e) {
  if (e == cudaSuccess) return vSuccess;
  (void)cudaGetLastError();
  return e == cudaErrorMemoryAllocation ? vOutOfMemory : vCudaError;
}

#define VC_TRY(x)                          \
  do {                                     \
    vResult_t r__ = fromCuda(x);           \
    if (r__ != vSuccess) return r__;       \
  } while (0)

int dtypeSize(int dt) { return (dt == kF16 || dt == kBF16) ? 2 : 4; }

size_t slotDataBytes(int proto, size_t slotBytes) {
  if (proto == kLL) return slotBytes / 2;             // 4 data bytes per 8-byte line
  if (proto == kLL128) return (slotBytes / 128) * 120; // 120 data bytes per 128-byte line
  return slotBytes;
}

// chunkCount in units: slot data x chunkSteps, whole 16-byte packs, >= 1 pack
unsigned long long chunkUnits(int proto, size_t slotBytes, int chunkSteps, int unitBytes) {
  unsigned long long epp = 16 / unitBytes;
  unsigned long long u = slotDataBytes(proto, slotBytes) * (unsigned long long)chunkSteps / unitBytes;
  u = u / epp * epp;
  return u < epp ? epp : u;
}

// occupancy cache: (kernel, threads) -> resident CTAs per SM
std::mutex gOccMu;
std::map<std::pair<const void*, int>, int> gOcc;

int residentPerSM(const void* fn, int nthr) {
  std::lock_guard<std::mutex> lk(gOccMu);
  auto key = std::make_pair(fn, nthr);
  auto it = gOcc.find(key);
  if (it != gOcc.end()) return it->second;
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, nthr, 0) != cudaSuccess) {
    (void)cudaGetLastError();
    nb = 0;
  }
  gOcc[key] = nb;
  return nb;
}

}  // namespace

struct vcomm {
  int k = 0, nch = 0, dev = 0, nsm = 0;
  size_t slotBytes[3] = {0, 0, 0};
  int nsteps = 8, nthreads = 1024;
  double timeoutSec = 5.0;
  Arena arena[2][3];
  ErrWord* hErr = nullptr;
  ErrWord* dErr = nullptr;
  int* dClaim = nullptr;
  int* hAbort = nullptr;
  int* dAbort = nullptr;
  bool pinned = false;
  vPlan_t pin{};
  vPlan_t last{};
};

static vResult_t freeComm(vcomm* c) {
  if (!c) return vSuccess;
  for (auto& row : c->arena)
    for (auto& a : row) {
      if (a.dConns) cudaFree(a.dConns);
      if (a.dBuf) cudaFree(a.dBuf);
      if (a.dCtr) cudaFree(a.dCtr);
    }
  if (c->dClaim) cudaFree(c->dClaim);
  if (c->hErr) cudaFreeHost(c->hErr);
  if (c->hAbort) cudaFreeHost(c->hAbort);
  (void)cudaGetLastError();
  delete c;
  return vSuccess;
}

static vResult_t ensureArena(vcomm* c, int algo, int proto) {
  Arena& a = c->arena[algo][proto];
  if (a.ready) return vSuccess;
  const int nsubMax = (algo == kTree) ? 2 * c->nch : c->nch;
  const int nconn = (algo == kTree) ? 2 * nsubMax * c->k : nsubMax * c->k;
  const size_t slot = c->slotBytes[proto];
  a.bytes = (size_t)nconn * (size_t)c->nsteps * slot;
  VC_TRY(cudaMalloc(&a.dBuf, a.bytes));
  VC_TRY(cudaMemset(a.dBuf, 0, a.bytes));
  const size_t ctrWords = (size_t)nconn * 2 * kCounterStride;
  VC_TRY(cudaMalloc(&a.dCtr, ctrWords * sizeof(unsigned long long)));
  VC_TRY(cudaMemset(a.dCtr, 0, ctrWords * sizeof(unsigned long long)));
  std::vector<ConnDev> h(nconn);
  for (int i = 0; i < nconn; i++) {
    h[i].buf = a.dBuf + (size_t)i * c->nsteps * slot;
    h[i].tail = a.dCtr + (size_t)(2 * i) * kCounterStride;
    h[i].head = a.dCtr + (size_t)(2 * i + 1) * kCounterStride;
    h[i].unused = 0;
  }
  VC_TRY(cudaMalloc(&a.dConns, nconn * sizeof(ConnDev)));
  VC_TRY(cudaMemcpy(a.dConns, h.data(), nconn * sizeof(ConnDev), cudaMemcpyHostToDevice));
  VC_TRY(cudaDeviceSynchronize());
  a.nconn = nconn;
  a.ready = true;
  return vSuccess;
}

extern "C" {

int vcommVersion(void) { return 100; }

vResult_t vcommInitConfig(vcomm_t* comm, int nranks, int nchannels, const vcommConfig_t* cfg) {
  if (!comm) return vInvalidArgument;
  *comm = nullptr;
  if (nranks < 1 || nranks > VCOMM_MAX_RANKS || nchannels < 1 || nchannels > VCOMM_MAX_CHANNELS)
    return vInvalidArgument;
  vcomm* c = new vcomm();
  c->k = nranks;
  c->nch = nchannels;
  for (int p = 0; p < 3; p++) {
    size_t s = (cfg && cfg->slotBytes[p]) ? cfg->slotBytes[p] : kDefaultSlot[p];
    if (s % 256 != 0 || s < 256) { delete c; return vInvalidArgument; }
    c->slotBytes[p] = s;
  }
  c->nsteps = (cfg && cfg->nsteps > 0) ? cfg->nsteps : 8;
  c->nthreads = (cfg && cfg->nthreads > 0) ? cfg->nthreads : 1024;
  if (c->nthreads % 64 != 0 || c->nthreads > 1024 || c->nsteps < 2 || c->nsteps > 64) {
    delete c;
    return vInvalidArgument;
  }
  c->timeoutSec = (cfg && cfg->timeoutSec > 0) ? cfg->timeoutSec : 5.0;
  if (!(cfg && cfg->timeoutSec > 0)) {
    const char* env = getenv("VCOMM_TIMEOUT_MS");
    if (env && atof(env) > 0) c->timeoutSec = atof(env) / 1000.0;
  }
  vResult_t r = fromCuda(cudaGetDevice(&c->dev));
  if (r == vSuccess) r = fromCuda(cudaDeviceGetAttribute(&c->nsm, cudaDevAttrMultiProcessorCount, c->dev));
  int coop = 0;
  if (r == vSuccess) r = fromCuda(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, c->dev));
  if (r == vSuccess && !coop) r = vUnsupported;
  if (r == vSuccess) r = fromCuda(cudaHostAlloc((void**)&c->hErr, sizeof(ErrWord), cudaHostAllocMapped));
  if (r == vSuccess) r = fromCuda(cudaHostGetDevicePointer((void**)&c->dErr, c->hErr, 0));
  if (r == vSuccess) r = fromCuda(cudaHostAlloc((void**)&c->hAbort, sizeof(int), cudaHostAllocMapped));
  if (r == vSuccess) r = fromCuda(cudaHostGetDevicePointer((void**)&c->dAbort, c->hAbort, 0));
  if (r == vSuccess) r = fromCuda(cudaMalloc(&c->dClaim, sizeof(int)));
  if (r == vSuccess) r = fromCuda(cudaMemset(c->dClaim, 0, sizeof(int)));
  if (r == vSuccess) r = fromCuda(cudaDeviceSynchronize());
  if (r != vSuccess) { freeComm(c); return r; }
  memset(c->hErr, 0, sizeof(ErrWord));
  *(volatile int*)c->hAbort = 0;
  *comm = c;
  return vSuccess;
}

vResult_t vcommInit(vcomm_t* comm, int nranks, int nchannels) {
  return vcommInitConfig(comm, nranks, nchannels, nullptr);
}

vResult_t vcommPrepare(vcomm_t c, unsigned algoMask, unsigned protoMask) {
  if (!c) return vInvalidArgument;
  for (int al = 0; al < 2; al++) {
    if (!(algoMask & (1u << (al + 1))) && !(algoMask & 1u)) continue;
    for (int p = 0; p < 3; p++) {
      if (!(protoMask & (1u << (p + 1))) && !(protoMask & 1u)) continue;
      vResult_t r = ensureArena(c, al, p);
      if (r != vSuccess) return r;
    }
  }
  return vSuccess;
}

vResult_t vcommDestroy(vcomm_t c) {
  if (!c) return vSuccess;
  vResult_t r = fromCuda(cudaDeviceSynchronize());
  freeComm(c);
  return r;
}

vResult_t vcommAbort(vcomm_t c) {
  if (!c) return vSuccess;
  *(volatile int*)c->hAbort = 1;
  vResult_t r = fromCuda(cudaDeviceSynchronize());
  freeComm(c);
  return r;
}

vResult_t vcommGetAsyncError(vcomm_t c, vResult_t* err) {
  if (!c || !err) return vInvalidArgument;
  *err = (vResult_t)((volatile ErrWord*)c->hErr)->code;
  return vSuccess;
}

vResult_t vcommSetPlan(vcomm_t c, const vPlan_t* plan) {
  if (!c) return vInvalidArgument;
  if (!plan) { c->pinned = false; return vSuccess; }
  if (plan->algo < vAlgoAuto || plan->algo > vAlgoTree || plan->proto < vProtoAuto ||
      plan->proto > vProtoLL128 || plan->nchannels < 0 || plan->nchannels > c->nch ||
      plan->chunkSteps < 0 || plan->chunkSteps > 64)
    return vInvalidArgument;
  c->pin = *plan;
  c->pinned = true;
  return vSuccess;
}

vResult_t vcommGetLastPlan(vcomm_t c, vPlan_t* plan) {
  if (!c || !plan) return vInvalidArgument;
  *plan = c->last;
  return vSuccess;
}

}  // extern "C"

// ------------------------------------------------------------------ planning
// Default tuning (used where neither the call nor a pin fixes a choice):
// LL below 64 KiB, LL128 below 2 MiB, Simple above (Sec. III-D: LL/LL128 for
// small messages, Simple for large); tree AllReduce up to 256 KiB (Sec. V-F:
// tree best for small, ring for large); about 1 MiB of message per channel.
static void defaultPlan(const vcomm* c, int coll, size_t bytes, vPlan_t* p) {
  if (p->proto == vProtoAuto) p->proto = bytes < (64u << 10) ? vProtoLL : bytes < (2u << 20) ? vProtoLL128 : vProtoSimple;
  if (p->algo == vAlgoAuto) p->algo = (coll == kAllReduce && bytes <= (256u << 10) && c->k > 2) ? vAlgoTree : vAlgoRing;
  if (p->nchannels <= 0) {
    size_t per = (size_t)1 << 20;
    size_t n = (bytes + per - 1) / per;
    if (p->algo == vAlgoTree) n = (n + 1) / 2;
    p->nchannels = (int)std::max<size_t>(1, std::min<size_t>(n, (size_t)c->nch));
  }
  if (p->chunkSteps <= 0) p->chunkSteps = 1;
}

// ------------------------------------------------------------------ one collective
static bool overlaps(uintptr_t a, size_t na, uintptr_t b, size_t nb) {
  return na && nb && a < b + nb && b < a + na;
}

static vResult_t collective(int coll, const void* const* sendbufs, void* const* recvbufs,
                            size_t count, int dtype, int op, int root, int algo, int proto,
                            vStream_t stream, vcomm_t c) {
  if (!c || !sendbufs || !recvbufs) return vInvalidArgument;
  {
    int e = ((volatile ErrWord*)c->hErr)->code;
    if (e != 0) return (vResult_t)e;   // a failed communicator stays failed
  }
  if (dtype < vInt32 || dtype > vBfloat16) return vInvalidArgument;
  if ((coll == kAllReduce || coll == kReduceScatter || coll == kReduce) && (op < vSum || op > vMax))
    return vInvalidArgument;
  if (algo < vAlgoAuto || algo > vAlgoTree || proto < vProtoAuto || proto > vProtoLL128)
    return vInvalidArgument;
  const int k = c->k;
  if ((coll == kBroadcast || coll == kReduce) && (root < 0 || root >= k)) return vInvalidArgument;
  if (algo == vAlgoTree && coll != kAllReduce) return vUnsupported;  // Table "collective support"
  if (count == 0) return vSuccess;
  const size_t esz = dtypeSize(dtype);

  // per-rank buffer sizes and which pointers are read / written
  size_t sb = count * esz, rb = count * esz;
  if (coll == kReduceScatter) sb = (size_t)k * count * esz;
  if (coll == kAllGather) rb = (size_t)k * count * esz;
  unsigned long long inplace = 0;
  for (int r = 0; r < k; r++) {
    const bool needSend = (coll != kBroadcast) || r == root;
    const bool needRecv = (coll != kReduce) || r == root;
    uintptr_t s = (uintptr_t)sendbufs[r], d = (uintptr_t)recvbufs[r];
    if ((needSend && !s) || (needRecv && !d)) return vInvalidArgument;
    if ((needSend && s % esz) || (needRecv && d % esz)) return vInvalidArgument;
    if (!needSend || !needRecv) continue;
    bool ip = false;
    if (coll == kAllGather) ip = (s == d + (size_t)r * sb);
    else if (coll == kReduceScatter) ip = (d == s + (size_t)r * rb);
    else ip = (s == d);
    if (ip) inplace |= 1ull << r;
    else if (overlaps(s, sb, d, rb)) return vInvalidArgument;
  }
  for (int r = 0; r < k; r++) {
    const bool needRecv = (coll != kReduce) || r == root;
    if (!needRecv) continue;
    uintptr_t d = (uintptr_t)recvbufs[r];
    for (int q = 0; q < k; q++) {
      if (q == r) continue;
      const bool qRecv = (coll != kReduce) || q == root;
      const bool qSend = (coll != kBroadcast) || q == root;
      if (qRecv && overlaps(d, rb, (uintptr_t)recvbufs[q], rb)) return vInvalidArgument;
      if (qSend && overlaps(d, rb, (uintptr_t)sendbufs[q], sb)) return vInvalidArgument;
    }
  }

  // plan
  vPlan_t plan{(vAlgo_t)algo, (vProto_t)proto, 0, 0};
  if (c->pinned) {
    if (plan.algo == vAlgoAuto) plan.algo = c->pin.algo;
    if (plan.proto == vProtoAuto) plan.proto = c->pin.proto;
    plan.nchannels = c->pin.nchannels;
    plan.chunkSteps = c->pin.chunkSteps;
  }
  if (plan.algo == vAlgoTree && coll != kAllReduce) plan.algo = vAlgoRing;
  defaultPlan(c, coll, std::max(sb, rb), &plan);
  int kcoll = coll;
  if (k == 1) {
    kcoll = kCopy;
    plan.algo = vAlgoRing;
    plan.proto = vProtoSimple;
  }
  // A ring FIFO step both receives and sends, and a slot is returned only
  // after the receiver's own send: if one chunk fills every slot of every
  // ring connection (chunkSteps >= nsteps), each rank waits for a credit from
  // its successor -- a cycle.  Ring collectives need chunkSteps < nsteps.
  if (plan.algo == vAlgoRing && k > 1 && plan.chunkSteps >= c->nsteps) {
    if (c->pinned && c->pin.chunkSteps > 0) return vUnsupported;
    plan.chunkSteps = c->nsteps - 1;
  }
  const int al = (plan.algo == vAlgoTree) ? kTree : kRing;
  const int pr = (int)plan.proto - 1;
  const bool bytesUnits = (coll == kAllGather || coll == kBroadcast);
  const void* fn = bytesUnits ? copyKernel(pr) : reduceKernel(pr, dtype, op < 0 ? 0 : op);
  if (!fn) return vInternalError;

  // co-residency: every CTA of the launch spins on its peers
  int nsub = (al == kTree) ? 2 * plan.nchannels : plan.nchannels;
  const int nthrMax = std::min(c->nthreads, maxThreadsFor(pr));
  int nthr = nthrMax;
  while (true) {
    int per = residentPerSM(fn, nthr);
    if ((long long)per * c->nsm >= (long long)k * nsub) break;
    if (nthr > 128) { nthr = (nthr / 2) / 64 * 64; continue; }
    // too many CTAs even with small blocks: shrink an automatic channel count
    bool autoCh = !(c->pinned && c->pin.nchannels > 0);
    if (autoCh && plan.nchannels > 1) {
      plan.nchannels--;
      nsub = (al == kTree) ? 2 * plan.nchannels : plan.nchannels;
      nthr = nthrMax;
      continue;
    }
    return vUnsupported;
  }

  if (kcoll != kCopy) {
    vResult_t r = ensureArena(c, al, pr);
    if (r != vSuccess) return r;
  }

  KernArgs a;
  memset(&a, 0, sizeof(a));
  for (int r = 0; r < k; r++) {
    a.send[r] = sendbufs[r];
    a.recv[r] = recvbufs[r];
  }
  const int unitBytes = bytesUnits ? 1 : (int)esz;
  if (coll == kAllGather || coll == kBroadcast) a.count = count * esz;
  else a.count = count;
  if (kcoll == kCopy && coll == kReduceScatter) a.count = count;  // block 0 of rank 0
  a.slotBytes = c->slotBytes[pr];
  a.slotUnits = slotDataBytes(pr, c->slotBytes[pr]) / unitBytes;
  a.chunk = chunkUnits(pr, c->slotBytes[pr], plan.chunkSteps, unitBytes);
  a.timeoutNs = (unsigned long long)(c->timeoutSec * 1e9);
  a.conns = (kcoll == kCopy) ? nullptr : c->arena[al][pr].dConns;
  a.errClaim = c->dClaim;
  a.err = c->dErr;
  a.abortFlag = c->dAbort;
  a.inplaceMask = inplace;
  a.downOffset = (unsigned long long)(2 * c->nch) * k;
  a.coll = kcoll;
  a.algo = al;
  a.nranks = k;
  a.nsub = nsub;
  a.root = root;
  a.nsteps = c->nsteps;
  a.upThreads = (nthr / 2) / 32 * 32;

  void* args[] = {(void*)&a};
  cudaError_t e = cudaLaunchCooperativeKernel(fn, dim3((unsigned)(k * nsub)), dim3((unsigned)nthr),
                                              args, 0, (cudaStream_t)stream);
  if (e != cudaSuccess) return fromCuda(e);
  c->last = plan;
  return vSuccess;
}

extern "C" {

vResult_t vAllReduce(const void* const* sendbufs, void* const* recvbufs, size_t count,
                     vDataType_t dtype, vRedOp_t op, vAlgo_t algo, vProto_t proto,
                     vStream_t stream, vcomm_t comm) {
  return collective(kAllReduce, sendbufs, recvbufs, count, dtype, op, 0, algo, proto, stream, comm);
}

vResult_t vReduceScatter(const void* const* sendbufs, void* const* recvbufs, size_t recvcount,
                         vDataType_t dtype, vRedOp_t op, vAlgo_t algo, vProto_t proto,
                         vStream_t stream, vcomm_t comm) {
  return collective(kReduceScatter, sendbufs, recvbufs, recvcount, dtype, op, 0, algo, proto,
                    stream, comm);
}

vResult_t vAllGather(const void* const* sendbufs, void* const* recvbufs, size_t sendcount,
                     vDataType_t dtype, vAlgo_t algo, vProto_t proto, vStream_t stream,
                     vcomm_t comm) {
  return collective(kAllGather, sendbufs, recvbufs, sendcount, dtype, -1, 0, algo, proto, stream,
                    comm);
}

vResult_t vBroadcast(const void* const* sendbufs, void* const* recvbufs, size_t count,
                     vDataType_t dtype, int root, vAlgo_t algo, vProto_t proto,
                     vStream_t stream, vcomm_t comm) {
  return collective(kBroadcast, sendbufs, recvbufs, count, dtype, -1, root, algo, proto, stream,
                    comm);
}

vResult_t vReduce(const void* const* sendbufs, void* const* recvbufs, size_t count,
                  vDataType_t dtype, vRedOp_t op, int root, vAlgo_t algo, vProto_t proto,
                  vStream_t stream, vcomm_t comm) {
  return collective(kReduce, sendbufs, recvbufs, count, dtype, op, root, algo, proto, stream, comm);
}

// ------------------------------------------------------------------ debug codecs
static std::mutex gDbgMu;
static int* gDbgClaim = nullptr;
static ErrWord* gDbgErrH = nullptr;
static ErrWord* gDbgErrD = nullptr;
static int* gDbgAbortH = nullptr;
static int* gDbgAbortD = nullptr;

vResult_t vDebugEncode(vProto_t proto, const void* src, size_t nbytes, uint64_t flag, void* lines,
                       vStream_t stream) {
  if (!src || !lines || (proto != vProtoLL && proto != vProtoLL128)) return vInvalidArgument;
  if (nbytes == 0) return vSuccess;
  const int p = (int)proto - 1;
  unsigned long long work = (p == kLL) ? (nbytes + 7) / 8 : 32 * (((nbytes + 119) / 120 + 3) / 4);
  unsigned blocks = (unsigned)std::min<unsigned long long>((work + 255) / 256, 4096);
  const char* s = (const char*)src;
  char* l = (char*)lines;
  unsigned long long nb = nbytes;
  void* args[] = {(void*)&p, (void*)&s, (void*)&nb, (void*)&flag, (void*)&l};
  return fromCuda(cudaLaunchKernel(debugEncodeKernel(), dim3(blocks), dim3(256), args, 0,
                                   (cudaStream_t)stream));
}

vResult_t vDebugDecode(vProto_t proto, const void* lines, size_t nbytes, uint64_t flag, void* dst,
                       double timeoutSec, vStream_t stream) {
  if (!lines || !dst || (proto != vProtoLL && proto != vProtoLL128)) return vInvalidArgument;
  if (nbytes == 0) return vSuccess;
  std::lock_guard<std::mutex> lk(gDbgMu);
  if (!gDbgClaim) {
    VC_TRY(cudaMalloc(&gDbgClaim, sizeof(int)));
    VC_TRY(cudaHostAlloc((void**)&gDbgErrH, sizeof(ErrWord), cudaHostAllocMapped));
    VC_TRY(cudaHostGetDevicePointer((void**)&gDbgErrD, gDbgErrH, 0));
    VC_TRY(cudaHostAlloc((void**)&gDbgAbortH, sizeof(int), cudaHostAllocMapped));
    VC_TRY(cudaHostGetDevicePointer((void**)&gDbgAbortD, gDbgAbortH, 0));
    *(volatile int*)gDbgAbortH = 0;
  }
  memset(gDbgErrH, 0, sizeof(ErrWord));
  VC_TRY(cudaMemsetAsync(gDbgClaim, 0, sizeof(int), (cudaStream_t)stream));
  KernArgs a;
  memset(&a, 0, sizeof(a));
  a.timeoutNs = (unsigned long long)((timeoutSec > 0 ? timeoutSec : 1.0) * 1e9);
  a.errClaim = gDbgClaim;
  a.err = gDbgErrD;
  a.abortFlag = gDbgAbortD;
  const int p = (int)proto - 1;
  unsigned long long work = (p == kLL) ? (nbytes + 7) / 8 : 32 * (((nbytes + 119) / 120 + 3) / 4);
  unsigned blocks = (unsigned)std::min<unsigned long long>((work + 255) / 256, 1024);
  const char* l = (const char*)lines;
  char* d = (char*)dst;
  unsigned long long nb = nbytes;
  void* args[] = {(void*)&a, (void*)&p, (void*)&l, (void*)&nb, (void*)&flag, (void*)&d};
  VC_TRY(cudaLaunchKernel(debugDecodeKernel(), dim3(blocks), dim3(256), args, 0, (cudaStream_t)stream));
  VC_TRY(cudaStreamSynchronize((cudaStream_t)stream));
  return (vResult_t)((volatile ErrWord*)gDbgErrH)->code;
}

}  // extern "C"
