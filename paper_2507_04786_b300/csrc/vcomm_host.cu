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
#include <cmath>
#include <memory>
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

int dtypeSize(int dt) {
  switch (dt) {
    case kI8: case kU8: return 1;
    case kF16: case kBF16: return 2;
    case kI64: case kU64: case kF64: return 8;
  }
  return 4;
}

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

constexpr int kTuneBuckets = 16;   // message sizes 1 KiB x 4^i

struct TuneEntry {
  bool valid = false;
  vPlan_t plan{};
  size_t bytes = 0;
  float usec = 0;
};

struct vcomm {
  int k = 0, nch = 0, dev = 0, nsm = 0;
  size_t slotBytes[3] = {0, 0, 0};
  int nsteps = 8, nthreads = 1024;
  double timeoutSec = 5.0;
  int treeNode = 1;                  // vranks per node of the hierarchical tree
  // direct AllReduce: bytes per rank from which the staged kernel runs
  unsigned long long stagedMinBytes = 8ull << 20;
  unsigned long long tileMinBytes = 64ull << 20;  // single calls the tile engine takes, from this size
  bool tileGroups = true;                     // groups of direct calls: one tile-engine launch
  Arena arena[2][3];
  ErrWord* hErr = nullptr;
  ErrWord* dErr = nullptr;
  int* dClaim = nullptr;
  int* hAbort = nullptr;
  int* dAbort = nullptr;
  bool pinned = false;
  vPlan_t pin{};
  vPlan_t last{};
  TuneEntry tune[5][kTuneBuckets];
  bool tuned[5] = {false, false, false, false, false};
  std::vector<vPlan_t> groupPlans;   // plans of the last group's calls, in call order
  int skipRank = -1;                 // fault injection (vcommDebugSetSkipRank)
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

// nesting depth of vGroupStart / vGroupEnd on this thread
static thread_local int tGroupDepth = 0;

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
  c->treeNode = (cfg && cfg->treeNodeSize > 0) ? cfg->treeNodeSize : 1;
  if (nranks % c->treeNode != 0) {
    delete c;
    return vInvalidArgument;
  }
  if (!(cfg && cfg->timeoutSec > 0)) {
    const char* env = getenv("VCOMM_TIMEOUT_MS");
    if (env && atof(env) > 0) c->timeoutSec = atof(env) / 1000.0;
  }
  if (const char* env = getenv("VCOMM_TILE_GROUPS")) c->tileGroups = !(env[0] == '0' && env[1] == 0);
  if (const char* env = getenv("VCOMM_STAGED_MIN_BYTES")) {
    char* end = nullptr;
    const unsigned long long v = strtoull(env, &end, 10);
    if (end && end != env && *end == 0) c->stagedMinBytes = v;
  }
  if (const char* env = getenv("VCOMM_TILE_MIN_BYTES")) {
    char* end = nullptr;
    const unsigned long long v = strtoull(env, &end, 10);
    if (end && end != env && *end == 0) c->tileMinBytes = v;
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

vResult_t vcommAbortPending(vcomm_t c) {
  if (!c) return vInvalidArgument;
  *(volatile int*)c->hAbort = 1;
  return fromCuda(cudaDeviceSynchronize());
}

vResult_t vcommReset(vcomm_t c) {
  if (!c) return vInvalidArgument;
  if (tGroupDepth > 0) return vInvalidArgument;
  VC_TRY(cudaDeviceSynchronize());   // nothing of this communicator may still run
  // a failed collective leaves its FIFOs half written and its counters
  // unequal: start every arena afresh
  for (auto& row : c->arena)
    for (auto& a : row) {
      if (!a.ready) continue;
      VC_TRY(cudaMemset(a.dBuf, 0, a.bytes));
      VC_TRY(cudaMemset(a.dCtr, 0, (size_t)a.nconn * 2 * kCounterStride * sizeof(unsigned long long)));
    }
  VC_TRY(cudaMemset(c->dClaim, 0, sizeof(int)));
  VC_TRY(cudaDeviceSynchronize());
  memset(c->hErr, 0, sizeof(ErrWord));
  *(volatile int*)c->hAbort = 0;
  c->skipRank = -1;
  return vSuccess;
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
      plan->proto > vProtoDirect || plan->nchannels < 0 || plan->nchannels > c->nch ||
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
// Default tuning (used where neither the call nor a pin fixes a choice and the
// communicator has not been tuned): the direct protocol on the ring (no FIFO
// at all: on one GPU it is the fastest at every size measured, 1 KiB to
// 256 MiB).  Where the caller asks for the tree, the FIFO protocols as the
// paper tunes them: up to 256 KiB the cluster protocol on <= 16 vranks (else
// LL below 64 KiB), LL128 below 2 MiB, Simple above (Sec. III-D); an Auto
// algorithm with a FIFO protocol takes the tree for AllReduce up to 256 KiB
// (Sec. V-F).  About 1 MiB of message per channel, 4 KiB for the cluster
// protocol (at most 64 / k clusters: a cluster of 16 CTAs takes most of a
// GPC).  A tuned communicator takes each Auto field from its measured table
// at the nearest size.
static void defaultPlan(const vcomm* c, int coll, size_t bytes, vPlan_t* p) {
  if (coll >= 0 && coll < 5 && c->tuned[coll]) {
    int best = -1;
    double bd = 1e30;
    for (int i = 0; i < kTuneBuckets; i++) {
      const TuneEntry& e = c->tune[coll][i];
      if (!e.valid) continue;
      double d = std::fabs(std::log2((double)e.bytes) - std::log2((double)std::max<size_t>(bytes, 1)));
      if (d < bd) { bd = d; best = i; }
    }
    if (best >= 0) {
      const vPlan_t& t = c->tune[coll][best].plan;
      const bool treeAsked = (p->algo == vAlgoTree);
      if (p->algo == vAlgoAuto) p->algo = t.algo;
      if (p->proto == vProtoAuto && !(treeAsked && t.proto == vProtoDirect)) p->proto = t.proto;
      if (p->nchannels <= 0) p->nchannels = std::min(t.nchannels, c->nch);
      if (p->chunkSteps <= 0) p->chunkSteps = t.chunkSteps;
    }
  }
  if (p->proto == vProtoAuto) {
    if (c->k >= 2 && p->algo != vAlgoTree) p->proto = vProtoDirect;
    else if (c->k >= 2 && c->k <= 16 && bytes <= (256u << 10)) p->proto = vProtoCluster;
    else p->proto = bytes < (64u << 10) ? vProtoLL : bytes < (2u << 20) ? vProtoLL128 : vProtoSimple;
  }
  if (p->algo == vAlgoAuto) {
    if (p->proto == vProtoDirect) p->algo = vAlgoRing;
    else p->algo = (coll == kAllReduce && bytes <= (256u << 10) && c->k > 2) ? vAlgoTree : vAlgoRing;
  }
  if (p->nchannels <= 0) {
    const bool cl = (p->proto == vProtoCluster);
    size_t per = cl ? ((size_t)4 << 10) : ((size_t)1 << 20);
    size_t n = (bytes + per - 1) / per;
    if (cl) n = std::min<size_t>(n, (size_t)std::max(1, 64 / c->k));
    if (p->algo == vAlgoTree) n = (n + 1) / 2;
    p->nchannels = (int)std::max<size_t>(1, std::min<size_t>(n, (size_t)c->nch));
  }
  if (p->chunkSteps <= 0) p->chunkSteps = 1;
}

// ------------------------------------------------------------------ one call
static bool overlaps(uintptr_t a, size_t na, uintptr_t b, size_t nb) {
  return na && nb && a < b + nb && b < a + na;
}

// everything a launch (single or batched) needs about one collective call
struct CallSpec {
  vcomm* c = nullptr;
  int coll = 0;                 // the user's collective
  int kcoll = 0;                // the kernel's (kCopy on a single rank)
  int dtype = 0, redop = 0, root = 0;
  int postDiv = 0;              // avg: k (the kernels add, the completing step divides)
  int al = 0, pr = 0;
  bool bytesUnits = false;
  vPlan_t plan{};
  unsigned long long units = 0; // partitioned units (0: nothing to do)
  unsigned long long inplace = 0;
  size_t S = 0;                 // the larger per-rank buffer, bytes
  int maxCtas = 0;              // direct protocol: cap on the grid (0: the whole GPU)
  cudaStream_t stream = nullptr;
  const void* send[VCOMM_MAX_RANKS];
  void* recv[VCOMM_MAX_RANKS];
};

static vResult_t prepareCall(int coll, const void* const* sendbufs, void* const* recvbufs,
                             size_t count, int dtype, int op, int root, int algo, int proto,
                             vStream_t stream, vcomm_t c, CallSpec* cs) {
  if (!c || !sendbufs || !recvbufs) return vInvalidArgument;
  {
    int e = ((volatile ErrWord*)c->hErr)->code;
    if (e != 0) return (vResult_t)e;   // a failed communicator stays failed
  }
  if (dtype < vInt32 || dtype > vFloat64) return vInvalidArgument;
  if ((coll == kAllReduce || coll == kReduceScatter || coll == kReduce) && (op < vSum || op > vAvg))
    return vInvalidArgument;
  if (algo < vAlgoAuto || algo > vAlgoTree || proto < vProtoAuto || proto > vProtoDirect)
    return vInvalidArgument;
  const int k = c->k;
  if ((coll == kBroadcast || coll == kReduce) && (root < 0 || root >= k)) return vInvalidArgument;
  if (algo == vAlgoTree && coll != kAllReduce) return vUnsupported;  // Table "collective support"
  cs->units = 0;
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
  if (plan.algo == vAlgoTree && (coll != kAllReduce || k < 2)) plan.algo = vAlgoRing;
  // the direct protocol replays ring fold orders only
  if (plan.proto == vProtoDirect && plan.algo == vAlgoTree) {
    if (algo == vAlgoTree || (c->pinned && c->pin.algo == vAlgoTree)) return vUnsupported;
    plan.algo = vAlgoRing;
  }
  int kcoll = coll;
  if (k == 1) {
    kcoll = kCopy;
    plan.algo = vAlgoRing;
    plan.proto = vProtoSimple;
  }
  // Ring Broadcast / Reduce chains on the FIFO protocols: with more CTAs
  // than SMs, two CTAs of the chains share an SM and the one waiting for its
  // predecessor spins beside the one moving data; at 16 vranks x 16 channels
  // a 128 MiB Broadcast took 4.7 ms against 1.6 ms at 9 channels.  The
  // channels are capped at (SMs / vranks); a chain's fold order does not
  // depend on the channels, so the results are the same.
  if ((coll == kBroadcast || coll == kReduce) && k > 1 &&
      (plan.proto == vProtoSimple || plan.proto == vProtoLL || plan.proto == vProtoLL128) &&
      (long long)k * plan.nchannels > c->nsm)
    plan.nchannels = std::max(1, c->nsm / k);
  // A ring FIFO step both receives and sends, and a slot is returned only
  // after the receiver's own send: if one chunk fills every slot of every
  // ring connection (chunkSteps >= nsteps), each rank waits for a credit from
  // its successor -- a cycle.  Ring collectives need chunkSteps < nsteps.
  // The cluster protocol (one cluster of k CTAs per channel) exists for
  // clusters of up to 16 CTAs, and its FIFOs have kClusterSlots slots.
  if (plan.proto == vProtoCluster && k > 16) return vUnsupported;
  const int fifoSlots = (plan.proto == vProtoCluster) ? kClusterSlots : c->nsteps;
  if (plan.algo == vAlgoRing && k > 1 && plan.proto != vProtoDirect && plan.chunkSteps >= fifoSlots) {
    if (c->pinned && c->pin.chunkSteps > 0) return vUnsupported;
    plan.chunkSteps = fifoSlots - 1;
  }
  cs->c = c;
  cs->coll = coll;
  cs->kcoll = kcoll;
  cs->dtype = dtype;
  cs->redop = op < 0 ? 0 : op;
  cs->postDiv = (op == vAvg && kcoll != kCopy) ? k : 0;
  cs->root = root;
  cs->al = (plan.algo == vAlgoTree) ? kTree : kRing;
  cs->pr = (int)plan.proto - 1;
  cs->bytesUnits = (coll == kAllGather || coll == kBroadcast);
  cs->plan = plan;
  cs->inplace = inplace;
  cs->S = std::max(sb, rb);
  cs->stream = (cudaStream_t)stream;
  if (cs->bytesUnits) cs->units = count * esz;
  else cs->units = count;
  for (int r = 0; r < k; r++) {
    cs->send[r] = sendbufs[r];
    cs->recv[r] = recvbufs[r];
  }
  return vSuccess;
}

static bool capturing(cudaStream_t s) {
  cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &st) != cudaSuccess) {
    (void)cudaGetLastError();
    return false;
  }
  return st != cudaStreamCaptureStatusNone;
}

// arenas are allocated outside stream capture only (cudaMalloc + sync)
static vResult_t needArena(vcomm* c, int al, int pr, cudaStream_t s) {
  if (c->arena[al][pr].ready) return vSuccess;
  if (capturing(s)) return vUnsupported;   // call vcommPrepare before capturing
  return ensureArena(c, al, pr);
}

// The cluster protocol: grid k * nsub CTAs in clusters of k (cluster = one
// channel, CTA r of it = vrank r), each with its FIFOs in dynamic shared
// memory.  Clusters never wait on one another, so no co-residency is needed
// beyond one cluster at a time, which the launch itself guarantees.
static vResult_t launchCluster(CallSpec& cs) {
  vcomm* c = cs.c;
  const int k = c->k;
  vPlan_t& plan = cs.plan;
  const void* fn = cs.bytesUnits ? clusterCopyKernel() : clusterKernel(cs.dtype, cs.redop);
  if (!fn) return vInternalError;
  {
    // once per kernel: opt in to the dynamic shared memory and to clusters
    // of more than 8 CTAs
    static std::mutex mu;
    static std::vector<const void*> ready;
    std::lock_guard<std::mutex> g(mu);
    if (std::find(ready.begin(), ready.end(), fn) == ready.end()) {
      VC_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, kClusterSmemBytes));
      VC_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
      ready.push_back(fn);
    }
  }
  const int nsub = (cs.al == kTree) ? 2 * plan.nchannels : plan.nchannels;
  const int nthr = std::min(c->nthreads, maxThreadsFor(kCluster));
  const int unitBytes = cs.bytesUnits ? 1 : dtypeSize(cs.dtype);

  KernArgs a;
  memset(&a, 0, sizeof(a));
  for (int r = 0; r < k; r++) {
    a.send[r] = cs.send[r];
    a.recv[r] = cs.recv[r];
  }
  a.count = cs.units;
  a.slotBytes = kClusterSlotBytes;
  a.slotUnits = (kClusterSlotBytes / 2) / unitBytes;
  a.chunk = chunkUnits(kLL, kClusterSlotBytes, plan.chunkSteps, unitBytes);
  a.timeoutNs = (unsigned long long)(c->timeoutSec * 1e9);
  a.conns = nullptr;
  a.errClaim = c->dClaim;
  a.err = c->dErr;
  a.abortFlag = c->dAbort;
  a.inplaceMask = cs.inplace;
  a.coll = cs.kcoll;
  a.algo = cs.al;
  a.redop = cs.redop;
  a.nranks = k;
  a.nsub = nsub;
  a.root = cs.root;
  a.nsteps = kClusterSlots;
  a.upThreads = (nthr / 2) / 32 * 32;
  a.skipRank = c->skipRank;
  a.postDiv = cs.postDiv;
  a.treeNode = c->treeNode;

  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(k * nsub));
  cfg.blockDim = dim3((unsigned)nthr);
  cfg.dynamicSmemBytes = kClusterSmemBytes;
  cfg.stream = cs.stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)k;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  {
    // does one cluster fit at all (k SMs of one GPC)?  Asked once per shape.
    static std::mutex mu;
    static std::map<std::pair<const void*, int>, int> fits;
    std::lock_guard<std::mutex> g(mu);
    auto key = std::make_pair(fn, k * 2048 + nthr);
    auto it = fits.find(key);
    if (it == fits.end()) {
      int fit = 0;
      VC_TRY(cudaOccupancyMaxActiveClusters(&fit, fn, &cfg));
      it = fits.emplace(key, fit).first;
    }
    if (it->second < 1) return vUnsupported;
  }
  void* args[] = {(void*)&a};
  VC_TRY(cudaLaunchKernelExC(&cfg, fn, args));
  c->last = plan;
  return vSuccess;
}

// Geometry of a direct call: whether every access can be a 16-byte vector
// (all buffers 16-byte aligned, and so the blocks inside them), the units
// the kernel spreads over its threads, and the Simple chunk that fixes the
// ring segments.
struct DirectGeom {
  int vec;                       // as DirectArgs::vec
  unsigned long long units, chunk;
};
static DirectGeom directGeom(const CallSpec& cs) {
  const int k = cs.c->k;
  const int esz = dtypeSize(cs.dtype);
  bool ptrs = true;
  for (int r = 0; r < k; r++)
    if (((uintptr_t)cs.send[r] | (uintptr_t)cs.recv[r]) & 15) ptrs = false;
  const bool wholeBlocks = !((cs.kcoll == kReduceScatter && (cs.units * esz) % 16) ||
                             (cs.kcoll == kAllGather && cs.units % 16));
  const unsigned long long chunk = chunkUnits(kSimple, cs.c->slotBytes[kSimple], cs.plan.chunkSteps, esz);
  if (ptrs && !wholeBlocks && cs.inplace == 0) {
    // blocks that are not whole 16-byte units: shifted 16-byte accesses
    const unsigned long long units = (cs.kcoll == kAllGather)
        ? cs.units * (unsigned long long)k / 16ull
        : (cs.units / (16ull / esz)) * (unsigned long long)k;
    return DirectGeom{2, units, chunk};
  }
  const bool aligned = ptrs && wholeBlocks;
  const unsigned long long per = aligned ? (cs.bytesUnits ? 16ull : 16ull / esz) : 1ull;
  unsigned long long units = cs.units / per;
  if (cs.kcoll == kReduceScatter || cs.kcoll == kAllGather) units *= (unsigned long long)k;
  return DirectGeom{aligned ? 1 : 0, units, chunk};
}

// The staged direct reducing kernel (bulk copies through shared memory)
// takes 16-byte aligned calls on the whole GPU from stagedMinBytes per rank
// (send buffer; 8 MiB, env VCOMM_STAGED_MIN_BYTES): AllReduce on 2..16
// vranks (fp64 up to 8), ReduceScatter and Reduce on 2..4 vranks, where a
// tile's one output leaves the register kernel ahead once the fold of more
// inputs, between two block barriers, outlasts the tile's loads.  Measured against the register kernel: smaller calls give a CTA
// too few tiles to fill the pipeline; beyond 16 vranks a tile holds fewer
// 16-byte units than the CTA has threads; fp64 folds of 16 vranks are bound
// by the fp64 pipe, where the register kernel's independent chains issue
// better.  Two stages of loads in flight suit up to 4 vranks, three more.
// The tile comes from directStagedTile for kStagedSmemMax bytes of shared
// memory.
constexpr int kStagedSmemMax = 205 * 1024;
static bool useStaged(const CallSpec& cs, const DirectGeom& g) {
  const int k = cs.c->k;
  const int kmax = cs.kcoll == kAllReduce ? 16 : (cs.kcoll == kReduceScatter || cs.kcoll == kReduce) ? 4 : 0;
  return g.vec == 1 && k >= 2 && k <= kmax && cs.maxCtas == 0 && !(cs.dtype == kF64 && k > 8) &&
         g.units * 16ull >= cs.c->stagedMinBytes;
}
static int stagedStages(int k) { return std::min(k <= 4 ? 2 : 3, directStagedMaxStages()); }
// Up to 3 vranks a tile's loads are too few bytes to keep HBM busy from one
// CTA per SM (k = 2: 3.3 TB/s); two CTAs per SM, each with half the shared
// memory, double them (k = 2: 5.2 TB/s).
static int stagedCtasPerSM(int k) { return k <= 3 ? 2 : 1; }

static vResult_t launchStaged(CallSpec& cs, const DirectGeom& g, DirectArgs& a) {
  vcomm* c = cs.c;
  const int k = c->k;
  const void* fn = directStagedKernel(cs.dtype, cs.redop);
  if (!fn) return vInternalError;
  {
    // once per kernel: opt in to the dynamic shared memory
    static std::mutex mu;
    static std::vector<const void*> ready;
    std::lock_guard<std::mutex> lk(mu);
    if (std::find(ready.begin(), ready.end(), fn) == ready.end()) {
      VC_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, kStagedSmemMax));
      ready.push_back(fn);
    }
  }
  const int stages = stagedStages(k);
  const int perSM = stagedCtasPerSM(k);
  const unsigned tile = directStagedTile(k, stages, kStagedSmemMax / perSM);
  const size_t smem = directStagedSmem(k, stages, tile);
  if (smem > (size_t)kStagedSmemMax) return vInternalError;
  a.stages = stages;
  a.tileBytes = tile;
  a.timeoutNs = (unsigned long long)(c->timeoutSec * 1e9);
  a.errClaim = c->dClaim;
  a.err = c->dErr;
  // tiles never straddle ReduceScatter blocks (g.units counts all k blocks)
  const unsigned long long nblk = cs.kcoll == kReduceScatter ? (unsigned long long)k : 1ull;
  const unsigned long long ntiles = nblk * ((g.units / nblk * 16ull + tile - 1) / tile);
  const long long grid = std::max<long long>(1, std::min<long long>((long long)ntiles, (long long)perSM * c->nsm));
  void* args[] = {(void*)&a};
  VC_TRY(cudaLaunchKernel(fn, dim3((unsigned)grid), dim3(directStagedThreads()), args, smem, cs.stream));
  c->last = cs.plan;
  return vSuccess;
}

// Copies staged through shared memory (AllGather, Broadcast and grouped
// point-to-point transfers): 16-byte aligned tasks whose sizes are multiples
// of 16 bytes, from stagedMinBytes per rank (AllGather, Broadcast) or in
// total (transfers), on the whole GPU.  Four stages of 32 KiB tiles, one CTA
// per SM.
constexpr unsigned kCopyTile = 32768;
constexpr int kCopyStages = 4;

static vResult_t launchCopyStaged(vcomm* c, CopyArgs& a, cudaStream_t stream) {
  const void* fn = copyStagedKernel();
  const int stages = std::min(kCopyStages, copyStagedMaxStages());
  const size_t smem = (size_t)stages * kCopyTile + 8 * (size_t)stages;
  {
    // once: opt in to the dynamic shared memory
    static std::mutex mu;
    static bool ready = false;
    std::lock_guard<std::mutex> lk(mu);
    if (!ready) {
      VC_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      ready = true;
    }
  }
  unsigned long long t = 0;
  for (int i = 0; i < a.ntasks; i++) {
    a.tasks[i].tileStart = t;
    t += (a.tasks[i].bytes + kCopyTile - 1) / kCopyTile;
  }
  a.ntiles = t;
  if (t == 0) return vSuccess;
  a.tile = (int)kCopyTile;
  a.stages = stages;
  a.timeoutNs = (unsigned long long)(c->timeoutSec * 1e9);
  a.errClaim = c->dClaim;
  a.err = c->dErr;
  const long long grid = std::max<long long>(1, std::min<long long>((long long)t, c->nsm));
  void* args[] = {(void*)&a};
  VC_TRY(cudaLaunchKernel(fn, dim3((unsigned)grid), dim3(32), args, smem, stream));
  return vSuccess;
}

// AllGather (one task per source rank) or Broadcast (one task) as staged
// copies, if the call qualifies
static bool useCopyStaged(const CallSpec& cs, const DirectGeom& g) {
  return (cs.kcoll == kAllGather || cs.kcoll == kBroadcast) && g.vec == 1 && cs.c->k >= 2 &&
         cs.maxCtas == 0 && cs.units % 16 == 0 && cs.units >= cs.c->stagedMinBytes;
}
static vResult_t launchCopyCollStaged(CallSpec& cs) {
  const int k = cs.c->k;
  CopyArgs a;
  memset(&a, 0, sizeof(a));
  for (int r = 0; r < k; r++) a.dsts[r] = cs.recv[r];
  if (cs.kcoll == kAllGather) {
    a.ntasks = k;
    for (int b = 0; b < k; b++) {
      CopyTask& t = a.tasks[b];
      t.src = cs.send[b];
      t.bytes = cs.units;
      t.dstOff = (unsigned long long)b * cs.units;
      t.skipMask = ((cs.inplace >> b) & 1ull) << b;
      t.dstBase = 0;
      t.ndst = k;
    }
  } else {
    a.ntasks = 1;
    CopyTask& t = a.tasks[0];
    t.src = cs.send[cs.root];
    t.bytes = cs.units;
    t.skipMask = ((cs.inplace >> cs.root) & 1ull) << cs.root;
    t.ndst = k;
  }
  const vResult_t r = launchCopyStaged(cs.c, a, cs.stream);
  if (r != vSuccess) return r;
  cs.c->last = cs.plan;
  return vSuccess;
}

static unsigned tileStageBytes(int dev);
static vResult_t launchTileGroup(vcomm* c, std::vector<CallSpec>& ops, unsigned stageBytes);

// Single calls that run faster as a one-call launch of the tile engine (a
// producer warp issuing bulk copies, eight consumer warps folding) than on
// the per-call kernels: AllReduce on 12..16 vranks (1.08-1.12x at 64 and 128
// MiB per rank) and ReduceScatter blocks that are not whole 16-byte units on
// up to 8 vranks (1.09-1.23x) -- from tileMinBytes per rank (send buffer;
// 64 MiB, env VCOMM_TILE_MIN_BYTES: at 32 MiB and below a CTA's one or two
// tiles leave the pipeline filling and draining, and the per-call kernels
// stay ahead), 32- and 16-bit types, sum or max.  Same fold, same bits.
static bool useTileEngine(const CallSpec& cs, const DirectGeom& g) {
  const int k = cs.c->k;
  if (!cs.c->tileGroups || cs.maxCtas != 0 || cs.postDiv || k < 2 || k > kServeMaxRanks) return false;
  if (!(cs.dtype == kI32 || cs.dtype == kF32 || cs.dtype == kF16 || cs.dtype == kBF16)) return false;
  if (!(cs.redop == kSum || cs.redop == kMax)) return false;
  const unsigned long long perRank =
      (cs.kcoll == kReduceScatter ? (unsigned long long)k : 1ull) * cs.units * (unsigned long long)dtypeSize(cs.dtype);
  if (perRank < cs.c->tileMinBytes) return false;
  if (cs.kcoll == kAllReduce) return g.vec == 1 && k >= 12;
  if (cs.kcoll == kReduceScatter) return g.vec == 2 && k <= 8;
  return false;
}

// The direct protocol: a plain launch over the data, no FIFO, no waits.
static vResult_t launchDirect(CallSpec& cs) {
  vcomm* c = cs.c;
  const int k = c->k;
  const void* fn = directKernel(cs.kcoll, cs.dtype, cs.redop);
  if (!fn) return vInternalError;
  const DirectGeom g = directGeom(cs);
  DirectArgs a;
  memset(&a, 0, sizeof(a));
  for (int r = 0; r < k; r++) {
    a.send[r] = cs.send[r];
    a.recv[r] = cs.recv[r];
  }
  a.count = cs.units;
  a.chunk = g.chunk;
  a.inplaceMask = cs.inplace;
  a.coll = cs.kcoll;
  a.nranks = k;
  a.nsub = cs.plan.nchannels;
  a.root = cs.root;
  a.vec = g.vec;
  a.postDiv = cs.postDiv;
  if (useTileEngine(cs, g)) {
    const unsigned sb = tileStageBytes(c->dev);
    if (sb) {
      std::vector<CallSpec> one{cs};
      const vResult_t r = launchTileGroup(c, one, sb);
      if (r == vSuccess) c->last = cs.plan;
      return r;
    }
  }
  if (useStaged(cs, g)) return launchStaged(cs, g, a);
  if (useCopyStaged(cs, g)) return launchCopyCollStaged(cs);
  const unsigned long long units = g.units;
  const int nthr = directThreads(cs.kcoll, cs.dtype);
  const long long resident = (long long)std::max(1, residentPerSM(fn, nthr)) * c->nsm;
  long long grid = (long long)((units + nthr - 1) / nthr);
  grid = std::max<long long>(1, std::min<long long>(grid, resident));
  if (cs.maxCtas > 0) grid = std::min<long long>(grid, cs.maxCtas);
  void* args[] = {(void*)&a};
  VC_TRY(cudaLaunchKernel(fn, dim3((unsigned)grid), dim3(nthr), args, 0, cs.stream));
  c->last = cs.plan;
  return vSuccess;
}

static vResult_t launchSingle(CallSpec& cs) {
  if (cs.pr == kCluster) return launchCluster(cs);
  if (cs.pr == kDirect) return launchDirect(cs);
  vcomm* c = cs.c;
  const int k = c->k;
  vPlan_t& plan = cs.plan;
  const void* fn = cs.bytesUnits ? copyKernel(cs.pr) : reduceKernel(cs.pr, cs.dtype, cs.redop);
  if (!fn) return vInternalError;

  // co-residency: every CTA of the launch spins on its peers
  int nsub = (cs.al == kTree) ? 2 * plan.nchannels : plan.nchannels;
  int nthrMax = std::min(c->nthreads, maxThreadsFor(cs.pr));
  // LL / LL128 on small calls: a step moves a few KiB, and a CTA of 256
  // threads turns its barriers and polls around faster than a full-size one
  // (16-vrank ring AllGather at 64 KiB per rank, LL: 49.9 -> 37.3 us against
  // 1024 threads, 26.4 -> 24.3 us against 512; 64 or 128 threads gain
  // nothing more); chains
  // and trees whose steps are larger keep the wider CTA (Broadcast of 64 KiB
  // over 8 channels: 16.2 us wide, 25.7 us narrow).  Same results.
  if (cs.pr == kLL || cs.pr == kLL128) {
    const unsigned long long unitB = cs.bytesUnits ? 1ull : (unsigned long long)dtypeSize(cs.dtype);
    // the larger buffer of a vrank: ReduceScatter's send, AllGather's receive
    const bool blocks = cs.kcoll == kReduceScatter || cs.kcoll == kAllGather;
    const unsigned long long perRank = (blocks ? (unsigned long long)k : 1ull) * cs.units * unitB;
    const unsigned long long perCh = perRank / (unsigned long long)std::max(1, plan.nchannels);
    const bool ringBlocks = cs.al == kRing && blocks;
    if ((ringBlocks && perRank <= (64ull << 10)) || perCh <= (4ull << 10)) nthrMax = std::min(nthrMax, 256);
  }
  int nthr = nthrMax;
  while (true) {
    int per = residentPerSM(fn, nthr);
    if ((long long)per * c->nsm >= (long long)k * nsub) break;
    if (nthr > 128) { nthr = (nthr / 2) / 64 * 64; continue; }
    // too many CTAs even with small blocks: shrink an automatic channel count
    bool autoCh = !(c->pinned && c->pin.nchannels > 0);
    if (autoCh && plan.nchannels > 1) {
      plan.nchannels--;
      nsub = (cs.al == kTree) ? 2 * plan.nchannels : plan.nchannels;
      nthr = nthrMax;
      continue;
    }
    return vUnsupported;
  }
  if (cs.kcoll != kCopy) {
    vResult_t r = needArena(c, cs.al, cs.pr, cs.stream);
    if (r != vSuccess) return r;
  }

  KernArgs a;
  memset(&a, 0, sizeof(a));
  for (int r = 0; r < k; r++) {
    a.send[r] = cs.send[r];
    a.recv[r] = cs.recv[r];
  }
  const int unitBytes = cs.bytesUnits ? 1 : dtypeSize(cs.dtype);
  a.count = cs.units;
  a.slotBytes = c->slotBytes[cs.pr];
  a.slotUnits = slotDataBytes(cs.pr, c->slotBytes[cs.pr]) / unitBytes;
  a.chunk = chunkUnits(cs.pr, c->slotBytes[cs.pr], plan.chunkSteps, unitBytes);
  a.timeoutNs = (unsigned long long)(c->timeoutSec * 1e9);
  a.conns = (cs.kcoll == kCopy) ? nullptr : c->arena[cs.al][cs.pr].dConns;
  a.errClaim = c->dClaim;
  a.err = c->dErr;
  a.abortFlag = c->dAbort;
  a.inplaceMask = cs.inplace;
  a.downOffset = (unsigned long long)(2 * c->nch) * k;
  a.coll = cs.kcoll;
  a.algo = cs.al;
  a.redop = cs.redop;
  a.nranks = k;
  a.nsub = nsub;
  a.root = cs.root;
  a.nsteps = c->nsteps;
  a.upThreads = (nthr / 2) / 32 * 32;
  a.skipRank = c->skipRank;
  a.postDiv = cs.postDiv;
  a.treeNode = c->treeNode;

  void* args[] = {(void*)&a};
  cudaError_t e = cudaLaunchCooperativeKernel(fn, dim3((unsigned)(k * nsub)), dim3((unsigned)nthr),
                                              args, 0, cs.stream);
  if (e != cudaSuccess) return fromCuda(e);
  c->last = plan;
  return vSuccess;
}

// ------------------------------------------------------------------ group calls
// vGroupStart / vGroupEnd (Sec. II-A-4): calls between them are validated and
// planned at once but launched together at vGroupEnd, one batch kernel per
// communicator.
static thread_local std::vector<CallSpec> tPending;

// ---- point-to-point (Sec. II-A-3: ncclSend / ncclRecv).  All vranks live in
// one process, so a transfer needs both sides inside one group; at
// vGroupEnd the k-th send from vrank a to b meets the k-th receive at b from
// a (order per ordered pair).  Same-process ranks move data with direct
// copies between source and destination buffers (Sec. IV, P2P_DIRECT); each
// transfer is its own task of one launch (Sec. II-C: grouped sends and
// receives run in parallel).
struct P2PSpec {
  vcomm* c;
  int rank, peer;
  bool send;
  const void* sbuf;
  void* rbuf;
  size_t bytes;
  int dtype;
  cudaStream_t stream;
};
static thread_local std::vector<P2PSpec> tP2P;

struct Transfer {
  const void* src;
  void* dst;
  size_t bytes;
};

// byte copies, one task each, as kDirectBatchCopy ops over one-rank views
static vResult_t launchCopies(vcomm* c, const std::vector<Transfer>& xs, cudaStream_t stream) {
  // staged copies when every transfer is 16-byte aligned and whole 16-byte
  // units and the group moves at least stagedMinBytes
  bool staged = !xs.empty();
  unsigned long long total = 0;
  for (const Transfer& t : xs) {
    if ((((uintptr_t)t.src | (uintptr_t)t.dst | t.bytes) & 15) != 0) staged = false;
    total += t.bytes;
  }
  if (staged && total >= c->stagedMinBytes) {
    for (size_t base = 0; base < xs.size(); base += kMaxCopyTasks) {
      const int n = (int)std::min<size_t>(kMaxCopyTasks, xs.size() - base);
      CopyArgs a;
      memset(&a, 0, sizeof(a));
      a.ntasks = n;
      for (int i = 0; i < n; i++) {
        const Transfer& x = xs[base + i];
        CopyTask& t = a.tasks[i];
        t.src = x.src;
        t.bytes = x.bytes;
        t.skipMask = x.src == x.dst ? 1ull : 0ull;
        t.dstBase = i;
        t.ndst = 1;
        a.dsts[i] = x.dst;
      }
      const vResult_t r = launchCopyStaged(c, a, stream);
      if (r != vSuccess) return r;
    }
    return vSuccess;
  }
  const void* fn = directBatchKernel(kBroadcast, 0, 0);
  const int nthr = directThreads(kBroadcast, 0);
  const long long resident = (long long)std::max(1, residentPerSM(fn, nthr)) * c->nsm;
  const int perLaunch = std::min<int>(kMaxBatchOps, kMaxBatchPtrs / 2);
  for (size_t base = 0; base < xs.size(); base += perLaunch) {
    const int n = (int)std::min<size_t>(perLaunch, xs.size() - base);
    std::unique_ptr<DirectBatchArgs> b(new DirectBatchArgs());
    memset(b.get(), 0, sizeof(DirectBatchArgs));
    b->nops = n;
    unsigned long long start = 0;
    for (int i = 0; i < n; i++) {
      const Transfer& t = xs[base + i];
      const bool vec = (((uintptr_t)t.src | (uintptr_t)t.dst) & 15) == 0;
      DirectOpDesc& d = b->ops[i];
      d.count = t.bytes;
      d.chunk = 16;
      d.inplaceMask = (t.src == t.dst) ? 1ull : 0ull;
      d.units = vec ? t.bytes / 16 : t.bytes;
      d.coll = kBroadcast;
      d.nranks = 1;
      d.nsub = 1;
      d.root = 0;
      d.vec = vec ? 1 : 0;
      d.ptrBase = 2 * i;
      b->ptrs[2 * i] = t.src;
      b->ptrs[2 * i + 1] = t.dst;
      b->unitStart[i] = start;
      start += std::max<unsigned long long>(d.units, 1ull);
    }
    b->unitStart[n] = start;
    long long grid = (long long)((start + nthr - 1) / nthr);
    grid = std::max<long long>(1, std::min<long long>(grid, resident));
    void* args[] = {(void*)b.get()};
    VC_TRY(cudaLaunchKernel(fn, dim3((unsigned)grid), dim3(nthr), args, 0, stream));
  }
  return vSuccess;
}

// match one communicator's sends and receives of a group into transfers
static vResult_t matchP2P(vcomm* c, const std::vector<P2PSpec>& ops, std::vector<Transfer>* out,
                          cudaStream_t* stream) {
  const int k = c->k;
  std::vector<std::vector<const P2PSpec*>> sends((size_t)k * k), recvs((size_t)k * k);
  for (auto& o : ops) {
    if (o.stream != ops[0].stream) return vInvalidArgument;   // one stream per group and comm
    if (o.send) sends[(size_t)o.rank * k + o.peer].push_back(&o);
    else recvs[(size_t)o.peer * k + o.rank].push_back(&o);
  }
  *stream = ops[0].stream;
  for (size_t pr = 0; pr < sends.size(); pr++) {
    if (sends[pr].size() != recvs[pr].size()) return vInvalidArgument;   // unmatched
    for (size_t i = 0; i < sends[pr].size(); i++) {
      const P2PSpec& a = *sends[pr][i];
      const P2PSpec& b = *recvs[pr][i];
      if (a.bytes != b.bytes || a.dtype != b.dtype) return vInvalidArgument;
      if (a.bytes) out->push_back(Transfer{a.sbuf, b.rbuf, a.bytes});
    }
  }
  return vSuccess;
}

// the direct calls of a group: one launch per (dtype, op) class present (one
// for the copies), each over up to kMaxBatchOps calls
// Shared memory per pipeline stage of the tile engine on this device: what
// the kernel's own shared memory and the output buffers leave of the
// largest opt-in, in three stages; 0 if the tile kernels cannot run.
static unsigned tileStageBytes(int dev) {
  static std::mutex mu;
  static std::map<int, unsigned> cache;
  std::lock_guard<std::mutex> lk(mu);
  auto it = cache.find(dev);
  if (it != cache.end()) return it->second;
  int maxSmem = 0;
  cudaFuncAttributes fa{};
  unsigned sb = 0;
  if (cudaDeviceGetAttribute(&maxSmem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) == cudaSuccess &&
      cudaFuncGetAttributes(&fa, batchTilesKernel()) == cudaSuccess) {
    const long long room = (long long)maxSmem - (long long)fa.sharedSizeBytes - (long long)serveTilesSmem(0);
    sb = room > 0 ? (unsigned)(room / serveTilesStages() / 128 * 128) : 0;
    if (sb < 16 * 128 ||
        cudaFuncSetAttribute(batchTilesKernel(), cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)serveTilesSmem(sb)) != cudaSuccess)
      sb = 0;
  }
  (void)cudaGetLastError();
  cache[dev] = sb;
  return sb;
}

// A group of direct calls as ONE launch of the tile engine (kBatchTiles):
// every call's tiles laid end to end, CTA j (one per SM) taking tiles j,
// j + grid, ...; 16-byte aligned AllReduce / ReduceScatter / AllGather tiles
// move by bulk copies through shared memory, the others take the register
// kernels' paths.  For calls of up to 16 vranks whose type and op the tile
// engine folds (int32, fp32, fp16, bf16; sum, max; copies); else false.
static bool tileBatchable(const vcomm* c, const std::vector<CallSpec>& ops) {
  if (c->k > kServeMaxRanks || ops.empty()) return false;
  for (const auto& o : ops) {
    if (o.kcoll != kAllReduce && o.kcoll != kReduceScatter && o.kcoll != kAllGather &&
        o.kcoll != kBroadcast && o.kcoll != kReduce)
      return false;
    if (o.postDiv) return false;
    const bool copy = (o.kcoll == kAllGather || o.kcoll == kBroadcast);
    if (!copy && !(o.dtype == kI32 || o.dtype == kF32 || o.dtype == kF16 || o.dtype == kBF16)) return false;
    if (!copy && !(o.redop == kSum || o.redop == kMax)) return false;
  }
  return true;
}

static vResult_t launchTileGroup(vcomm* c, std::vector<CallSpec>& ops, unsigned stageBytes) {
  const int k = c->k;
  const cudaStream_t stream = ops[0].stream;
  for (size_t base = 0; base < ops.size(); base += kMaxBatchOps) {
    const int n = (int)std::min<size_t>(kMaxBatchOps, ops.size() - base);
    std::unique_ptr<TileBatchArgs> b(new TileBatchArgs());
    memset(b.get(), 0, sizeof(TileBatchArgs));
    b->nops = n;
    b->stageBytes = stageBytes;
    b->copyTimeoutNs = (unsigned long long)(c->timeoutSec * 1e9);
    b->errClaim = c->dClaim;
    b->err = c->dErr;
    // the tiles are shared out statically (CTA j takes j, j + grid, ...):
    // ops in order of falling traffic per tile, so that every round of
    // `grid` tiles holds tiles of about one size and the CTAs finish together
    struct OpTiles {
      int idx;
      DirectGeom g;
      TileGeometry tg;
      unsigned long long perTile;
    };
    std::vector<OpTiles> order;
    for (int i = 0; i < n; i++) {
      const CallSpec& o = ops[base + i];
      OpTiles t{i, directGeom(o), {}, 0};
      const int esz = dtypeSize(o.dtype);
      t.tg = tileGeometry(o.kcoll, k, o.units, esz, t.g.vec, (unsigned long long)c->nsm,
                          (unsigned long long)serveTilesUnitsPerIter(), true);
      const bool copy = o.kcoll == kAllGather || o.kcoll == kBroadcast;
      const unsigned long long factor = o.kcoll == kAllReduce ? 2ull * k : (unsigned long long)k + 1;
      const unsigned long long unitBytes = t.tg.vec == 0 ? (copy ? 1ull : (unsigned long long)esz) : 16ull;
      t.perTile = (t.tg.staged ? t.tg.tileBytes : t.tg.tileUnits * unitBytes) * factor;
      order.push_back(t);
    }
    std::stable_sort(order.begin(), order.end(),
                     [](const OpTiles& a, const OpTiles& b) { return a.perTile > b.perTile; });
    unsigned long long start = 0;
    for (int i = 0; i < n; i++) {
      const CallSpec& o = ops[base + order[i].idx];
      const DirectGeom& g = order[i].g;
      const TileGeometry& tg = order[i].tg;
      TileOpDesc& d = b->ops[i];
      d.count = o.units;
      d.chunk = g.chunk;
      d.inplaceMask = o.inplace;
      d.staged = tg.staged;
      d.units = tg.units;
      d.tileUnits = tg.tileUnits;
      d.blockBytes = tg.blockBytes;
      d.tileBytes = tg.tileBytes;
      d.perBlock = tg.perBlock;
      d.ntiles = tg.ntiles;
      d.tileStart = start;
      d.coll = o.kcoll;
      d.dtype = o.dtype;
      d.redop = o.redop;
      d.nranks = k;
      d.nsub = o.plan.nchannels;
      d.root = o.root;
      d.vec = tg.vec;
      d.ptrBase = 2 * k * i;
      for (int r = 0; r < k; r++) {
        b->ptrs[d.ptrBase + r] = o.send[r];
        b->ptrs[d.ptrBase + k + r] = o.recv[r];
      }
      start += tg.ntiles;
    }
    b->totalTiles = start;
    const unsigned grid = (unsigned)std::max<unsigned long long>(1, std::min<unsigned long long>(start, c->nsm));
    void* args[] = {(void*)b.get()};
    VC_TRY(cudaLaunchKernel(batchTilesKernel(), dim3(grid), dim3(serveTilesThreads()), args,
                            serveTilesSmem(stageBytes), stream));
  }
  return vSuccess;
}

static vResult_t launchDirectGroup(vcomm* c, std::vector<CallSpec>& ops) {
  const int k = c->k;
  const cudaStream_t stream = ops[0].stream;
  if (c->tileGroups && tileBatchable(c, ops)) {
    const unsigned sb = tileStageBytes(c->dev);
    if (sb) return launchTileGroup(c, ops, sb);
  }
  const int perLaunch = std::min<int>(kMaxBatchOps, kMaxBatchPtrs / (2 * k));
  const int kCopyClass = kNumDtypes * kNumOps;
  auto classOf = [&](const CallSpec& o) {
    return (o.kcoll == kAllGather || o.kcoll == kBroadcast) ? kCopyClass : o.dtype * kNumOps + o.redop;
  };
  for (int cls = 0; cls <= kCopyClass; cls++) {
    std::vector<const CallSpec*> mine;
    for (auto& o : ops)
      if (classOf(o) == cls) mine.push_back(&o);
    if (mine.empty()) continue;
    const CallSpec& first = *mine[0];
    const void* fn = directBatchKernel(first.kcoll, first.dtype, first.redop);
    const int nthr = directThreads(first.kcoll, first.dtype);
    const long long resident = (long long)std::max(1, residentPerSM(fn, nthr)) * c->nsm;
    for (size_t base = 0; base < mine.size(); base += perLaunch) {
      const int n = (int)std::min<size_t>(perLaunch, mine.size() - base);
      std::unique_ptr<DirectBatchArgs> b(new DirectBatchArgs());
      memset(b.get(), 0, sizeof(DirectBatchArgs));
      b->nops = n;
      unsigned long long start = 0;
      for (int i = 0; i < n; i++) {
        const CallSpec& o = *mine[base + i];
        const DirectGeom g = directGeom(o);
        DirectOpDesc& d = b->ops[i];
        d.count = o.units;
        d.chunk = g.chunk;
        d.inplaceMask = o.inplace;
        d.units = g.units;
        d.coll = o.kcoll;
        d.nranks = k;
        d.nsub = o.plan.nchannels;
        d.root = o.root;
        d.dtype = o.dtype;
        d.redop = o.redop;
        d.vec = g.vec;
        d.postDiv = o.postDiv;
        d.ptrBase = 2 * k * i;
        for (int r = 0; r < k; r++) {
          b->ptrs[d.ptrBase + r] = o.send[r];
          b->ptrs[d.ptrBase + k + r] = o.recv[r];
        }
        b->unitStart[i] = start;
        start += std::max<unsigned long long>(g.units, 1ull);   // a unit range to own the tail
      }
      b->unitStart[n] = start;
      long long grid = (long long)((start + nthr - 1) / nthr);
      grid = std::max<long long>(1, std::min<long long>(grid, resident));
      void* args[] = {(void*)b.get()};
      VC_TRY(cudaLaunchKernel(fn, dim3((unsigned)grid), dim3(nthr), args, 0, stream));
    }
  }
  return vSuccess;
}

static vResult_t launchFifoGroup(vcomm* c, std::vector<CallSpec>& ops);

// launch a group: its direct calls in one direct batch launch, the FIFO
// calls in one persistent batch kernel (or a plain launch if alone)
static vResult_t launchGroup(vcomm* c, std::vector<CallSpec>& ops) {
  if (ops.empty()) return vSuccess;
  const cudaStream_t stream = ops[0].stream;
  for (auto& o : ops)
    if (o.stream != stream) return vInvalidArgument;   // one stream per group and communicator
  if (ops.size() == 1) {
    vResult_t r = launchSingle(ops[0]);
    c->groupPlans.assign(1, ops[0].plan);
    return r;
  }
  std::vector<CallSpec> direct, fifo;
  std::vector<std::pair<int, int>> where;   // (0 direct / 1 fifo, index)
  for (auto& o : ops) {
    if (o.pr == kDirect && o.kcoll != kCopy) {
      where.emplace_back(0, (int)direct.size());
      direct.push_back(o);
    } else {
      where.emplace_back(1, (int)fifo.size());
      fifo.push_back(o);
    }
  }
  vResult_t r = vSuccess;
  if (!direct.empty()) r = launchDirectGroup(c, direct);
  if (r == vSuccess && fifo.size() == 1) r = launchSingle(fifo[0]);
  else if (r == vSuccess && fifo.size() > 1) r = launchFifoGroup(c, fifo);
  if (r != vSuccess) return r;
  c->groupPlans.clear();
  for (auto& w : where) c->groupPlans.push_back(w.first == 0 ? direct[w.second].plan : fifo[w.second].plan);
  c->last = ops.back().plan;
  return vSuccess;
}

// launch the FIFO calls of a group: gangs, LPT assignment, one kernel
static vResult_t launchFifoGroup(vcomm* c, std::vector<CallSpec>& ops) {
  const cudaStream_t stream = ops[0].stream;
  const int k = c->k;
  const void* fn = batchKernel();
  const int nthr = 256;
  const int resident = residentPerSM(fn, nthr) * c->nsm;
  // gangs: up to 4 concurrent op streams, each on nch / G channels
  int G = std::min<int>(std::min<int>(4, (int)ops.size()), c->nch);
  int cpg = c->nch / G;
  while ((long long)G * k * cpg > resident) {
    if (cpg > 1) cpg--;
    else if (G > 1) { G--; cpg = c->nch / G; }
    else return vUnsupported;
  }
  // fit each op's plan into a gang (the batch kernel has no cluster
  // protocol: such ops run as LL)
  for (auto& o : ops) {
    if (o.pr == kCluster) { o.pr = kLL; o.plan.proto = vProtoLL; }
    if (o.pr == kDirect) { o.pr = kSimple; o.plan.proto = vProtoSimple; }   // single-rank copies
    if (o.kcoll == kCopy) {
      o.plan.nchannels = std::min(o.plan.nchannels, cpg);
      continue;
    }
    if (o.al == kTree && cpg < 2) { o.al = kRing; o.plan.algo = vAlgoRing; }
    if (o.al == kTree) o.plan.nchannels = std::min(o.plan.nchannels, cpg / 2);
    else o.plan.nchannels = std::min(o.plan.nchannels, cpg);
    if (o.al == kRing && k > 1 && o.plan.chunkSteps >= c->nsteps) o.plan.chunkSteps = c->nsteps - 1;
    vResult_t r = needArena(c, o.al, o.pr, stream);
    if (r != vSuccess) return r;
  }

  // launches of at most kMaxBatchOps ops and kMaxBatchPtrs pointers each
  const int perLaunch = std::min<int>(kMaxBatchOps, kMaxBatchPtrs / (2 * k));
  for (size_t base = 0; base < ops.size(); base += perLaunch) {
    const int n = (int)std::min<size_t>(perLaunch, ops.size() - base);
    // longest-processing-time-first assignment by a bytes-moved cost model
    std::vector<int> idx(n);
    std::vector<double> cost(n);
    for (int i = 0; i < n; i++) {
      const CallSpec& o = ops[base + i];
      const double f = (o.pr == kLL) ? 2.0 : (o.pr == kLL128) ? 128.0 / 120.0 : 1.0;
      cost[i] = (double)o.S * f + 65536.0;   // + a per-op latency in byte-equivalents
      idx[i] = i;
    }
    std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) { return cost[a] > cost[b]; });
    std::vector<double> load(G, 0.0);
    std::vector<int> gangOf(n);
    for (int i : idx) {
      int g = (int)(std::min_element(load.begin(), load.end()) - load.begin());
      gangOf[i] = g;
      load[g] += cost[i];
    }
    std::unique_ptr<BatchArgs> b(new BatchArgs());
    memset(b.get(), 0, sizeof(BatchArgs));
    b->timeoutNs = (unsigned long long)(c->timeoutSec * 1e9);
    b->errClaim = c->dClaim;
    b->err = c->dErr;
    b->abortFlag = c->dAbort;
    b->nops = n;
    b->nranks = k;
    b->ngangs = G;
    b->cpg = cpg;
    b->nsteps = c->nsteps;
    b->treeNode = c->treeNode;
    int pos = 0;
    for (int g = 0; g < G; g++) {
      b->gangStart[g] = pos;
      for (int i = 0; i < n; i++)   // submission order inside a gang
        if (gangOf[i] == g) b->order[pos++] = (unsigned char)i;
    }
    b->gangStart[G] = pos;
    for (int i = 0; i < n; i++) {
      const CallSpec& o = ops[base + i];
      BatchOpDesc& d = b->ops[i];
      const int unitBytes = o.bytesUnits ? 1 : dtypeSize(o.dtype);
      d.count = o.units;
      d.chunk = chunkUnits(o.pr, c->slotBytes[o.pr], o.plan.chunkSteps, unitBytes);
      d.slotBytes = c->slotBytes[o.pr];
      d.slotUnits = slotDataBytes(o.pr, c->slotBytes[o.pr]) / unitBytes;
      d.inplaceMask = o.inplace;
      d.downOffset = (unsigned long long)(2 * c->nch) * k;
      d.conns = (o.kcoll == kCopy) ? nullptr : c->arena[o.al][o.pr].dConns;
      d.coll = o.kcoll;
      d.algo = o.al;
      d.proto = o.pr;
      d.dtype = o.bytesUnits ? -1 : o.dtype;
      d.redop = o.redop;
      d.nsub = (o.al == kTree) ? 2 * o.plan.nchannels : o.plan.nchannels;
      d.root = o.root;
      d.postDiv = o.postDiv;
      d.ptrBase = 2 * k * i;
      for (int r = 0; r < k; r++) {
        b->ptrs[2 * k * i + r] = o.send[r];
        b->ptrs[2 * k * i + k + r] = o.recv[r];
      }
    }
    void* args[] = {(void*)b.get()};
    cudaError_t e = cudaLaunchCooperativeKernel(fn, dim3((unsigned)(G * k * cpg)), dim3(nthr), args, 0,
                                                stream);
    if (e != cudaSuccess) return fromCuda(e);
  }
  c->last = ops.back().plan;
  return vSuccess;
}

// the serving layer's launch: a ring collective whose direct-protocol grid
// is capped at maxCtas, so that concurrent requests on other streams keep
// SMs (other protocols ignore the cap); returns the plan it ran
vResult_t vc::serveCollective(int coll, const void* const* sendbufs, void* const* recvbufs, size_t count,
                              int dtype, int op, int proto, void* stream, vcomm_t c, int maxCtas,
                              vPlan_t* plan) {
  CallSpec cs;
  vResult_t r = prepareCall(coll, sendbufs, recvbufs, count, dtype, op, 0, vAlgoRing, proto, stream, c, &cs);
  if (r != vSuccess) return r;
  if (plan) *plan = cs.plan;
  if (cs.units == 0) return vSuccess;
  cs.maxCtas = maxCtas;
  return launchSingle(cs);
}

static vResult_t collective(int coll, const void* const* sendbufs, void* const* recvbufs,
                            size_t count, int dtype, int op, int root, int algo, int proto,
                            vStream_t stream, vcomm_t c) {
  CallSpec cs;
  vResult_t r = prepareCall(coll, sendbufs, recvbufs, count, dtype, op, root, algo, proto, stream,
                            c, &cs);
  if (r != vSuccess || cs.units == 0) return r;
  if (tGroupDepth > 0) {
    tPending.push_back(cs);
    c->last = cs.plan;
    return vSuccess;
  }
  return launchSingle(cs);
}

// ------------------------------------------------------------------ tuner
// Measures every candidate plan (algorithm, protocol, channels) at message
// sizes 1 KiB x 4^i up to maxBytes, on scratch buffers, with CUDA events on
// the caller's stream, and keeps the fastest per size: the table that
// defaultPlan consults (Sec. III-D / V-F: the choice depends on size).
static const int kTuneColls[5] = {kAllReduce, kReduceScatter, kAllGather, kBroadcast, kReduce};

static vResult_t tuneOne(vcomm* c, int coll, size_t S, char* sbuf, char* rbuf, size_t stride,
                         cudaStream_t s, cudaEvent_t e0, cudaEvent_t e1) {
  const int k = c->k;
  size_t count = S / 4;
  if (coll == kReduceScatter || coll == kAllGather) count = S / 4 / k;
  if (count == 0) return vSuccess;
  std::vector<const void*> sp(k);
  std::vector<void*> rp(k);
  for (int r = 0; r < k; r++) {
    sp[r] = sbuf + (size_t)r * stride;
    rp[r] = rbuf + (size_t)r * stride;
  }
  std::vector<int> chans;
  for (int ch : {1, 2, 4, 8, 16, 32, 64})
    if (ch <= c->nch) chans.push_back(ch);
  if (std::find(chans.begin(), chans.end(), c->nch) == chans.end()) chans.push_back(c->nch);
  TuneEntry best{};
  best.usec = 1e30f;
  const bool savedPinned = c->pinned;
  const vPlan_t savedPin = c->pin;
  for (int al = 0; al < ((coll == kAllReduce && k > 2) ? 2 : 1); al++) {
    for (int pr = 0; pr < 5; pr++) {
      // the cluster protocol is a small-message protocol on <= 16 vranks;
      // the direct protocol replays ring orders only
      if (pr == kCluster && (k > 16 || S > ((size_t)4 << 20))) continue;
      if (pr == kDirect && al == 1) continue;
      for (int ch : chans) {
        vPlan_t p{al ? vAlgoTree : vAlgoRing, (vProto_t)(pr + 1), ch, 1};
        c->pin = p;
        c->pinned = true;
        CallSpec cs;
        vResult_t r = prepareCall(coll, sp.data(), rp.data(), count, vFloat32, vSum, 0, p.algo,
                                  p.proto, s, c, &cs);
        if (r == vSuccess && cs.units) r = launchSingle(cs);   // warm-up (and arena)
        if (r != vSuccess) { (void)cudaGetLastError(); continue; }
        const int reps = 3;
        cudaEventRecord(e0, s);
        for (int i = 0; i < reps && r == vSuccess; i++) r = launchSingle(cs);
        cudaEventRecord(e1, s);
        if (cudaEventSynchronize(e1) != cudaSuccess || r != vSuccess) {
          (void)cudaGetLastError();
          continue;
        }
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        const float us = ms * 1000.0f / reps;
        if (us < best.usec) {
          best.valid = true;
          best.usec = us;
          best.bytes = S;
          best.plan = cs.plan;
        }
      }
    }
  }
  c->pinned = savedPinned;
  c->pin = savedPin;
  int bucket = 0;
  while (((size_t)1024 << (2 * bucket)) < S && bucket < kTuneBuckets - 1) bucket++;
  if (best.valid) {
    c->tune[coll][bucket] = best;
    c->tuned[coll] = true;
  }
  int e = ((volatile ErrWord*)c->hErr)->code;
  return e ? (vResult_t)e : vSuccess;
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

static vResult_t p2pCall(bool send, const void* sbuf, void* rbuf, size_t count, vDataType_t dtype,
                         int rank, int peer, vcomm_t c, vStream_t stream) {
  if (!c || dtype < vInt32 || dtype > vFloat64) return vInvalidArgument;
  if (rank < 0 || rank >= c->k || peer < 0 || peer >= c->k) return vInvalidArgument;
  const size_t esz = dtypeSize(dtype);
  const void* p = send ? sbuf : rbuf;
  if (count && (!p || (uintptr_t)p % esz)) return vInvalidArgument;
  if (tGroupDepth <= 0) return vInvalidArgument;   // both sides must be in one group
  {
    int e = ((volatile ErrWord*)c->hErr)->code;
    if (e != 0) return (vResult_t)e;
  }
  tP2P.push_back(P2PSpec{c, rank, peer, send, sbuf, rbuf, count * esz, (int)dtype, (cudaStream_t)stream});
  return vSuccess;
}

vResult_t vSend(const void* sendbuf, size_t count, vDataType_t dtype, int rank, int peer, vcomm_t comm,
                vStream_t stream) {
  return p2pCall(true, sendbuf, nullptr, count, dtype, rank, peer, comm, stream);
}

vResult_t vRecv(void* recvbuf, size_t count, vDataType_t dtype, int rank, int peer, vcomm_t comm,
                vStream_t stream) {
  return p2pCall(false, nullptr, recvbuf, count, dtype, rank, peer, comm, stream);
}

vResult_t vAllToAll(const void* const* sendbufs, void* const* recvbufs, size_t count, vDataType_t dtype,
                    vcomm_t c, vStream_t stream) {
  if (!c || !sendbufs || !recvbufs || dtype < vInt32 || dtype > vFloat64) return vInvalidArgument;
  const int k = c->k;
  const size_t esz = dtypeSize(dtype), blk = count * esz;
  for (int r = 0; r < k; r++) {
    if (count && (!sendbufs[r] || !recvbufs[r])) return vInvalidArgument;
    if ((uintptr_t)sendbufs[r] % esz || (uintptr_t)recvbufs[r] % esz) return vInvalidArgument;
    // a receive buffer may not overlap any buffer but (exactly) its own send buffer
    for (int q = 0; q < k && count; q++) {
      if (q != r && overlaps((uintptr_t)recvbufs[r], k * blk, (uintptr_t)recvbufs[q], k * blk))
        return vInvalidArgument;
      if (overlaps((uintptr_t)recvbufs[r], k * blk, (uintptr_t)sendbufs[q], k * blk) &&
          !(q == r && recvbufs[r] == sendbufs[r] && k == 1))
        return vInvalidArgument;
    }
  }
  {
    int e = ((volatile ErrWord*)c->hErr)->code;
    if (e != 0) return (vResult_t)e;
  }
  if (count == 0) return vSuccess;
  // the grouped send / receive pattern of Sec. II-A-4: rank r's block j goes
  // to block r of rank j
  if (tGroupDepth > 0) {
    for (int r = 0; r < k; r++)
      for (int j = 0; j < k; j++) {
        const char* s = (const char*)sendbufs[r] + (size_t)j * blk;
        char* d = (char*)recvbufs[j] + (size_t)r * blk;
        tP2P.push_back(P2PSpec{c, r, j, true, s, nullptr, blk, (int)dtype, (cudaStream_t)stream});
        tP2P.push_back(P2PSpec{c, j, r, false, nullptr, d, blk, (int)dtype, (cudaStream_t)stream});
      }
    return vSuccess;
  }
  std::vector<Transfer> xs;
  for (int r = 0; r < k; r++)
    for (int j = 0; j < k; j++)
      xs.push_back(Transfer{(const char*)sendbufs[r] + (size_t)j * blk, (char*)recvbufs[j] + (size_t)r * blk, blk});
  return launchCopies(c, xs, (cudaStream_t)stream);
}

vResult_t vcommDebugSetSkipRank(vcomm_t c, int rank) {
  if (!c || rank < -1 || rank >= c->k) return vInvalidArgument;
  c->skipRank = rank;
  return vSuccess;
}

vResult_t vGroupStart(void) {
  tGroupDepth++;
  return vSuccess;
}

vResult_t vGroupEnd(void) {
  if (tGroupDepth <= 0) return vInvalidArgument;
  if (--tGroupDepth > 0) return vSuccess;
  std::vector<CallSpec> pending;
  pending.swap(tPending);
  std::vector<P2PSpec> p2p;
  p2p.swap(tP2P);
  // one batch per communicator, in order of first appearance
  vResult_t first = vSuccess;
  std::vector<vcomm*> comms;
  for (auto& o : pending)
    if (std::find(comms.begin(), comms.end(), o.c) == comms.end()) comms.push_back(o.c);
  for (auto& o : p2p)
    if (std::find(comms.begin(), comms.end(), o.c) == comms.end()) comms.push_back(o.c);
  // every communicator's sends and receives must match before anything runs
  std::vector<std::vector<Transfer>> xfers(comms.size());
  std::vector<cudaStream_t> xstream(comms.size(), nullptr);
  for (size_t i = 0; i < comms.size(); i++) {
    std::vector<P2PSpec> mine;
    for (auto& o : p2p)
      if (o.c == comms[i]) mine.push_back(o);
    if (mine.empty()) continue;
    vResult_t r = matchP2P(comms[i], mine, &xfers[i], &xstream[i]);
    if (r != vSuccess) return r;
  }
  for (size_t i = 0; i < comms.size(); i++) {
    vcomm* c = comms[i];
    std::vector<CallSpec> ops;
    for (auto& o : pending)
      if (o.c == c) ops.push_back(o);
    vResult_t r = ops.empty() ? vSuccess : launchGroup(c, ops);
    if (r == vSuccess && !xfers[i].empty()) r = launchCopies(c, xfers[i], xstream[i]);
    if (r != vSuccess && first == vSuccess) first = r;
  }
  return first;
}

vResult_t vcommGetGroupPlans(vcomm_t c, vPlan_t* plans, int maxPlans, int* nPlans) {
  if (!c || !nPlans || maxPlans < 0 || (maxPlans > 0 && !plans)) return vInvalidArgument;
  const int n = (int)c->groupPlans.size();
  for (int i = 0; i < n && i < maxPlans; i++) plans[i] = c->groupPlans[i];
  *nPlans = n;
  return vSuccess;
}

vResult_t vcommTune(vcomm_t c, unsigned collMask, size_t maxBytes, vStream_t stream) {
  if (!c || maxBytes < 1024 || maxBytes > ((size_t)1 << 34)) return vInvalidArgument;
  if (tGroupDepth > 0) return vInvalidArgument;
  cudaStream_t s = (cudaStream_t)stream;
  if (capturing(s)) return vUnsupported;
  const size_t stride = (maxBytes + 255) / 256 * 256;
  char* sbuf = nullptr;
  char* rbuf = nullptr;
  VC_TRY(cudaMalloc(&sbuf, stride * c->k));
  vResult_t r = fromCuda(cudaMalloc(&rbuf, stride * c->k));
  if (r == vSuccess) r = fromCuda(cudaMemset(sbuf, 0, stride * c->k));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (r == vSuccess) r = fromCuda(cudaEventCreate(&e0));
  if (r == vSuccess) r = fromCuda(cudaEventCreate(&e1));
  for (int ci = 0; ci < 5 && r == vSuccess; ci++) {
    if (!(collMask & (1u << ci))) continue;
    for (size_t S = 1024; S <= maxBytes && r == vSuccess; S *= 4)
      r = tuneOne(c, kTuneColls[ci], S, sbuf, rbuf, stride, s, e0, e1);
  }
  cudaStreamSynchronize(s);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(sbuf);
  if (rbuf) cudaFree(rbuf);
  (void)cudaGetLastError();
  return r;
}

vResult_t vcommGetTuneTable(vcomm_t c, int coll, vPlan_t* plans, size_t* bytes, float* usec,
                            int maxEntries, int* nEntries) {
  if (!c || !nEntries || coll < 0 || coll > 4 || maxEntries < 0) return vInvalidArgument;
  int n = 0;
  for (int i = 0; i < kTuneBuckets; i++) {
    const TuneEntry& e = c->tune[kTuneColls[coll]][i];
    if (!e.valid) continue;
    if (n < maxEntries) {
      if (plans) plans[n] = e.plan;
      if (bytes) bytes[n] = e.bytes;
      if (usec) usec[n] = e.usec;
    }
    n++;
  }
  *nEntries = n;
  return vSuccess;
}

// ------------------------------------------------------------------ debug: tile geometry
vResult_t vDebugTileGeometry(int coll, int nranks, unsigned long long count, int dtypeSize, int vec,
                             unsigned long long workers, unsigned long long iter, int shared,
                             unsigned long long* out) {
  if (!out || coll < kAllReduce || coll > kReduce || nranks < 1 || nranks > kServeMaxRanks ||
      !(dtypeSize == 1 || dtypeSize == 2 || dtypeSize == 4) || vec < 0 || vec > 2 || iter == 0)
    return vInvalidArgument;
  const TileGeometry g = tileGeometry(coll, nranks, count, dtypeSize, vec, workers, iter, shared != 0);
  out[0] = g.staged;
  out[1] = g.units;
  out[2] = g.tileUnits;
  out[3] = g.blockBytes;
  out[4] = g.tileBytes;
  out[5] = g.perBlock;
  out[6] = g.ntiles;
  out[7] = (unsigned long long)g.vec;
  return vSuccess;
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
  a.skipRank = -1;
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
