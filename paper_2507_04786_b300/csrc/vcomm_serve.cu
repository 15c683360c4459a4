// vcomm_serve.cu -- serving: continuous batching of collective requests.
//
// Requests (AllReduce / ReduceScatter / AllGather over 1..16 vranks) arrive
// at any time.  A host dispatch thread admits them in arrival order, letting
// later ones pass a request that has to wait, as soon as (a) the bytes of all
// admitted, unreleased requests stay within the device-memory budget and (b)
// a gang of the persistent serving kernel is free; it carves the request's
// output buffers out of the budget pool, posts the request to the gang's
// host-mapped mailbox and timestamps the completion the gang reports.  Gangs
// run concurrently, so requests overlap on the device; one wide gang takes the
// large requests, narrow gangs the small ones.  A request's plan (protocol,
// channels, chunk) depends only on the request, so its result is the same
// alone and in any mix.  Mode "plain" runs the same stream of requests as one
// ordinary collective launch each, on one stream, for comparison; mode
// "streams" launches each request on a lane of streams; mode "tiles" (the
// direct protocol only) posts each admitted request to a ring in host-mapped
// memory that one resident tile-engine kernel ingests, its CTAs taking the
// requests' tiles from device queues (vcomm_serve_tiles.cu).
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstddef>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "vcomm.h"
#include "vcomm_internal.h"
#include "vcomm_kernels.h"

using namespace vc;

namespace {

int64_t nowNs() {
  return std::chrono::duration_cast<std::chrono::nanoseconds>(
             std::chrono::steady_clock::now().time_since_epoch()).count();
}

vResult_t fromCudaS(cudaError_t e) {
  if (e == cudaSuccess) return vSuccess;
  (void)cudaGetLastError();
  return e == cudaErrorMemoryAllocation ? vOutOfMemory : vCudaError;
}

size_t slotData(int proto, size_t slotBytes) {
  if (proto == kLL) return slotBytes / 2;
  if (proto == kLL128) return (slotBytes / 128) * 120;
  return slotBytes;
}

// first-fit allocator over the budget pool (host bookkeeping only)
struct Pool {
  size_t size = 0;
  std::map<size_t, size_t> free_;   // offset -> bytes
  void init(size_t n) { size = n; free_.clear(); if (n) free_[0] = n; }
  bool alloc(size_t n, size_t* off) {
    n = (n + 255) / 256 * 256;
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= n) {
        *off = it->first;
        size_t rest = it->second - n, o2 = it->first + n;
        free_.erase(it);
        if (rest) free_[o2] = rest;
        return true;
      }
    }
    return false;
  }
  void release(size_t off, size_t n) {
    n = (n + 255) / 256 * 256;
    auto it = free_.emplace(off, n).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }
};

struct Request {
  uint64_t ticket = 0;
  int coll = 0, dtype = 0, redop = 0, nranks = 0, flags = 0;
  vProto_t proto = vProtoAuto;
  size_t count = 0, sb = 0, rb = 0;   // per-rank send / recv bytes
  const void* send[kServeMaxRanks] = {};
  void* recv[kServeMaxRanks] = {};
  size_t poolOff[kServeMaxRanks] = {};
  int64_t arrivalNs = 0, doneNs = 0, serviceNs = -1;
  int state = 0;                      // 0 queued, 1 running, 2 done, 3 failed
  int gang = -1;
  bool big = false;
  vPlan_t plan{};
  cudaEvent_t ev = nullptr;           // modes 1, 2: end of the request's launch
  cudaEvent_t ev0 = nullptr;          // modes 1, 2: start of the request's launch
  int lane = -1;                      // mode 2: the stream it runs on
  uint64_t tseq = 0;                  // mode 3: its sequence number in the request ring
};

}  // namespace

struct vserve {
  vserveConfig_t cfg{};
  int dev = 0, nsm = 0;
  cudaStream_t stream = nullptr;
  char* pool = nullptr;
  Pool alloc;
  size_t inflight = 0, maxInflight = 0;
  // continuous-batching mode
  int ngangs = 0;
  std::vector<int> gangCpg;
  ServeSlot* hSlots = nullptr;
  ServeSlot* dSlots = nullptr;
  ServeGang* dGangs = nullptr;
  int* hShutdown = nullptr;
  int* dShutdown = nullptr;
  ErrWord* hErr = nullptr;
  ErrWord* dErr = nullptr;
  int* hAbort = nullptr;
  int* dAbort = nullptr;
  int* dClaim = nullptr;
  char* arenaBuf[3] = {nullptr, nullptr, nullptr};
  unsigned long long* arenaCtr[3] = {nullptr, nullptr, nullptr};
  ConnDev* arenaConns[3] = {nullptr, nullptr, nullptr};
  std::vector<uint64_t> posted;       // per gang: requests posted
  std::vector<uint64_t> running;      // per gang: ticket running (0: free)
  bool kernelUp = false;
  // plain mode (and the communicators of mode 2)
  vcomm_t comms[kServeMaxRanks + 1] = {};
  std::deque<uint64_t> plainInflight;
  // stream mode: lane 0 for large requests, lanes 1.. for the others; each
  // lane's launches are capped at laneCtas[l] CTAs so that the lanes overlap
  std::vector<cudaStream_t> lanes;
  std::vector<int> laneCtas;
  std::vector<std::deque<uint64_t>> laneInflight;
  // a FIFO-protocol launch on comms[k] waits for the previous one (the
  // arena of a communicator serves one call at a time; lanes are streams)
  cudaEvent_t commEv[kServeMaxRanks + 1] = {};
  bool commEvUsed[kServeMaxRanks + 1] = {};
  // tiles mode (3): the request ring, completions and control words
  // (host-mapped), the kernel's device state, and the host's view of them
  TileReq* hRing = nullptr;
  TileReq* dRing = nullptr;
  TileDone* hDone = nullptr;
  TileDone* dDone = nullptr;
  TileCtl* hCtl = nullptr;
  TileCtl* dCtl = nullptr;
  TileState* dState = nullptr;
  TileQueues* dQueues = nullptr;
  cudaEvent_t tilesEnd = nullptr;     // recorded after every launch of the tile kernel
  bool tilesUp = false;
  int tileWorkers = 0;
  unsigned tileStageBytes = 0;
  uint64_t tilePosted = 0;            // requests written to the ring (sequence numbers 0, 1, ...)
  std::vector<uint64_t> tileTicket;   // ring entry -> ticket of its request (0: free)
  std::deque<uint64_t> tileInflight;  // tickets posted, not completed
  // requests
  std::mutex mu;
  std::deque<uint64_t> incoming;      // submitted, not yet seen by the dispatcher
  std::deque<uint64_t> bigQ;          // seen, not admitted: large requests (wide gang)
  std::deque<uint64_t> smallQ;        // seen, not admitted: the others
  std::unordered_map<uint64_t, Request> reqs;
  uint64_t nextTicket = 1;
  uint64_t submitted = 0, completed = 0, failed = 0;
  std::thread th;
  std::atomic<bool> stop{false};
  vResult_t threadErr = vSuccess;
};

namespace {

// the plan of a request depends on the request alone (see the file comment)
void planFor(const vserve* s, Request& q) {
  const size_t S = std::max(q.sb, q.rb);
  vProto_t p = q.proto;
  // Auto: the direct protocol (no FIFO), the fastest at every size on one GPU
  if (p == vProtoAuto) p = vProtoDirect;
  q.big = S >= s->cfg.bigThreshold;
  // a request spreads over its whole gang: channels = gang CTAs / vranks
  // (mode 1: over up to 2 CTAs per SM), at most ~1 MiB of message per channel
  const int ctas = (s->cfg.mode == 0) ? (q.big ? s->gangCpg[0] : 1) * s->cfg.maxRanks
                                      : std::min(2 * s->nsm, q.nranks * VCOMM_MAX_CHANNELS);
  // (modes 1, 2 and 3 share this rule, so their plans and results agree)
  size_t per = (size_t)1 << 20;
  int ch = (int)std::max<size_t>(1, std::min<size_t>((S + per - 1) / per,
                                                      (size_t)std::max(1, ctas / q.nranks)));
  q.plan = vPlan_t{vAlgoRing, p, ch, 1};
}

// Kernels are loaded on their first launch; a server that launches per
// request would otherwise pay that (milliseconds) inside the latency of its
// first requests of every kind.  Looking up a kernel's attributes loads it.
void preloadKernels(int mode) {
  std::vector<const void*> fns;
  for (int dt = vInt32; dt <= vBfloat16; dt++) {
    for (int op = vSum; op <= vMax; op++) {
      for (int coll : {kAllReduce, kReduceScatter, kAllGather}) fns.push_back(directKernel(coll, dt, op));
      fns.push_back(directStagedKernel(dt, op));
      if (mode == 1 || mode == 2)
        for (int p = 0; p < 3; p++) fns.push_back(reduceKernel(p, dt, op));
    }
  }
  fns.push_back(copyStagedKernel());
  if (mode == 1 || mode == 2)
    for (int p = 0; p < 3; p++) fns.push_back(copyKernel(p));
  for (const void* f : fns) {
    cudaFuncAttributes fa;
    if (f && cudaFuncGetAttributes(&fa, f) != cudaSuccess) (void)cudaGetLastError();
  }
}

void completeReq(vserve* s, Request& q, bool ok) {
  q.doneNs = nowNs();
  q.state = ok ? 2 : 3;
  if (ok) s->completed++;
  else s->failed++;
  if (q.flags & 1) {   // release the outputs at completion
    for (int r = 0; r < q.nranks; r++)
      if (q.recv[r]) s->alloc.release(q.poolOff[r], q.rb);
    s->inflight -= (q.sb + q.rb) * q.nranks;
    for (int r = 0; r < q.nranks; r++) q.recv[r] = nullptr;
  }
}

bool allocOutputs(vserve* s, Request& q) {
  int r = 0;
  for (; r < q.nranks; r++) {
    size_t off;
    if (!s->alloc.alloc(q.rb, &off)) break;
    q.poolOff[r] = off;
    q.recv[r] = s->pool + off;
  }
  if (r == q.nranks) return true;
  for (int i = 0; i < r; i++) s->alloc.release(q.poolOff[i], q.rb);
  for (int i = 0; i < q.nranks; i++) q.recv[i] = nullptr;
  return false;
}

void postToGang(vserve* s, Request& q, int g) {
  ServeReq sr;
  memset(&sr, 0, sizeof(sr));
  const int pr = (int)q.plan.proto - 1;
  const bool bytes = (q.coll == kAllGather);
  const int unitBytes = bytes ? 1 : ((q.dtype == vFloat16 || q.dtype == vBfloat16) ? 2 : 4);
  const size_t esz = (q.dtype == vFloat16 || q.dtype == vBfloat16) ? 2 : 4;
  sr.coll = (q.nranks == 1) ? kCopy : q.coll;
  sr.proto = (q.nranks == 1) ? kSimple : pr;
  sr.dtype = bytes ? -1 : q.dtype;
  if (sr.proto == kDirect) {
    // no FIFO: the gang's CTAs fold the units from the user buffers; the
    // segments (fold order) come from the Simple slot's chunk, as in a plain call
    sr.dtype = q.dtype;
    sr.redop = q.redop;
    sr.nranks = q.nranks;
    sr.nsub = q.plan.nchannels;
    sr.count = bytes ? q.count * esz : q.count;
    unsigned long long epp = 16 / unitBytes;
    unsigned long long ch = s->cfg.slotBytes[kSimple] * (unsigned long long)q.plan.chunkSteps / unitBytes;
    ch = ch / epp * epp;
    sr.chunk = ch < epp ? epp : ch;
    bool aligned = true;
    for (int r = 0; r < q.nranks; r++) {
      sr.send[r] = q.send[r];
      sr.recv[r] = q.recv[r];
      if (((uintptr_t)q.send[r] | (uintptr_t)q.recv[r]) & 15) aligned = false;
    }
    if (q.coll == kReduceScatter && (q.count * esz) % 16) aligned = false;
    if (q.coll == kAllGather && (q.count * esz) % 16) aligned = false;
    sr.vec = aligned ? 1 : 0;
  } else {
  sr.redop = q.redop;
  sr.nranks = q.nranks;
  sr.nsub = q.plan.nchannels;
  sr.root = 0;
  sr.count = bytes ? q.count * esz : q.count;
  const size_t slotB = s->cfg.slotBytes[sr.proto];
  sr.slotBytes = slotB;
  sr.slotUnits = slotData(sr.proto, slotB) / unitBytes;
  unsigned long long epp = 16 / unitBytes;
  unsigned long long ch = slotData(sr.proto, slotB) * (unsigned long long)q.plan.chunkSteps / unitBytes;
  ch = ch / epp * epp;
  sr.chunk = ch < epp ? epp : ch;
  sr.inplaceMask = 0;
  for (int r = 0; r < q.nranks; r++) {
    sr.send[r] = q.send[r];
    sr.recv[r] = q.recv[r];
  }
  }
  volatile ServeSlot* slot = &s->hSlots[g];
  memcpy((void*)&slot->req, &sr, sizeof(sr));
  std::atomic_thread_fence(std::memory_order_seq_cst);
  s->posted[g]++;
  slot->seq = s->posted[g];
  std::atomic_thread_fence(std::memory_order_seq_cst);
  s->running[g] = q.ticket;
  q.gang = g;
  q.state = 1;
}

// mode 3: (re)start the tile kernel; it ingests from ring sequence firstSeq on
vResult_t launchTiles(vserve* s, uint64_t firstSeq) {
  volatile TileCtl* ctl = s->hCtl;
  if (ctl->error) return (vResult_t)ctl->error;   // a failed kernel is not restarted
  ctl->stopped = 0;
  ctl->shutdown = 0;
  std::atomic_thread_fence(std::memory_order_seq_cst);
  vResult_t r = fromCudaS(cudaMemsetAsync(&s->dQueues->stop, 0, sizeof(int), s->stream));
  if (r != vSuccess) return r;
  TileArgs a;
  memset(&a, 0, sizeof(a));
  a.ring = s->dRing;
  a.done = s->dDone;
  a.ctl = s->dCtl;
  a.state = s->dState;
  a.q = s->dQueues;
  a.firstSeq = firstSeq;
  a.idleTimeoutNs = (unsigned long long)(s->cfg.idleTimeoutSec * 1e9);
  a.drainTimeoutNs = 5000000000ull;
  a.copyTimeoutNs = 5000000000ull;
  a.stageBytes = s->tileStageBytes;
  void* args[] = {(void*)&a};
  r = fromCudaS(cudaLaunchCooperativeKernel(serveTilesKernel(), dim3(1 + s->tileWorkers),
                                            dim3(serveTilesThreads()), args,
                                            serveTilesSmem(s->tileStageBytes), s->stream));
  if (r != vSuccess) return r;
  r = fromCudaS(cudaEventRecord(s->tilesEnd, s->stream));
  if (r == vSuccess) s->tilesUp = true;
  return r;
}

// mode 3: the tile kernel has returned (idle, or stopped): requests it took
// and finished are reported by the completion scan; the ones it never took
// are taken by the next launch
void noteTilesExit(vserve* s) {
  if (!s->tilesUp) return;
  cudaError_t e = cudaEventQuery(s->tilesEnd);
  if (e == cudaErrorNotReady) return;
  (void)cudaGetLastError();
  s->tilesUp = false;
}

// mode 3: write request q into the ring (false: its ring entry is still busy)
bool postTile(vserve* s, Request& q) {
  const uint64_t seq = s->tilePosted;
  const int slot = (int)(seq % kTileRing);
  if (s->tileTicket[slot]) return false;
  noteTilesExit(s);
  if (!s->tilesUp) {
    // the kernel went idle: start it again at the first request it has not taken
    const uint64_t from = *(volatile unsigned long long*)&s->hCtl->ingested;
    if (launchTiles(s, from) != vSuccess) return false;
  }
  TileReq tr;
  memset(&tr, 0, sizeof(tr));
  ServeReq& sr = tr.req;
  const size_t esz = (q.dtype == vFloat16 || q.dtype == vBfloat16) ? 2 : 4;
  const bool copy = (q.coll == kAllGather);
  sr.coll = q.coll;
  sr.proto = kDirect;
  sr.dtype = q.dtype;
  sr.redop = q.redop;
  sr.nranks = q.nranks;
  sr.nsub = q.plan.nchannels;
  sr.count = copy ? q.count * esz : q.count;
  // the segments (fold order) come from the Simple slot's chunk, as in a plain call
  const unsigned long long unitBytes = copy ? 1 : esz;
  const unsigned long long epp = 16 / unitBytes;
  unsigned long long ch = s->cfg.slotBytes[kSimple] * (unsigned long long)q.plan.chunkSteps / unitBytes;
  ch = ch / epp * epp;
  sr.chunk = ch < epp ? epp : ch;
  bool ptrs = true;
  for (int r = 0; r < q.nranks; r++) {
    sr.send[r] = q.send[r];
    sr.recv[r] = q.recv[r];
    if (((uintptr_t)q.send[r] | (uintptr_t)q.recv[r]) & 15) ptrs = false;
  }
  const bool whole = !((q.coll == kReduceScatter || q.coll == kAllGather) && (q.count * esz) % 16);
  // 1: 16-byte units; 2: aligned buffers, blocks not whole units (shifted
  // 16-byte accesses, register path); 0: element accesses
  sr.vec = ptrs ? (whole ? 1 : 2) : 0;
  const TileGeometry tg = tileGeometry(q.coll, q.nranks, sr.count, (int)esz, sr.vec,
                                      (unsigned long long)s->tileWorkers,
                                      (unsigned long long)serveTilesUnitsPerIter());
  sr.vec = tg.vec;
  tr.staged = tg.staged;
  tr.units = tg.units;
  tr.tileUnits = tg.tileUnits;
  tr.blockBytes = tg.blockBytes;
  tr.tileBytes = tg.tileBytes;
  tr.perBlock = tg.perBlock;
  tr.ntiles = tg.ntiles;
  tr.klass = q.big ? 1 : 0;
  volatile TileReq* dst = &s->hRing[slot];
  memcpy((void*)dst, &tr, offsetof(TileReq, seq));
  std::atomic_thread_fence(std::memory_order_seq_cst);
  dst->seq = seq + 1;
  std::atomic_thread_fence(std::memory_order_seq_cst);
  s->tileTicket[slot] = q.ticket;
  s->tilePosted = seq + 1;
  s->tileInflight.push_back(q.ticket);
  q.tseq = seq;
  q.gang = slot;
  q.state = 1;
  return true;
}

vResult_t launchPlain(vserve* s, Request& q) {
  vcomm_t c = s->comms[q.nranks];
  if (!q.ev0) cudaEventCreate(&q.ev0);
  cudaEventRecord(q.ev0, s->stream);
  vcommSetPlan(c, &q.plan);
  vResult_t r;
  if (q.coll == kAllReduce)
    r = vAllReduce(q.send, q.recv, q.count, (vDataType_t)q.dtype, (vRedOp_t)q.redop, vAlgoRing,
                   q.plan.proto, s->stream, c);
  else if (q.coll == kReduceScatter)
    r = vReduceScatter(q.send, q.recv, q.count, (vDataType_t)q.dtype, (vRedOp_t)q.redop, vAlgoRing,
                       q.plan.proto, s->stream, c);
  else
    r = vAllGather(q.send, q.recv, q.count, (vDataType_t)q.dtype, vAlgoRing, q.plan.proto,
                   s->stream, c);
  if (r != vSuccess) return r;
  vcommGetLastPlan(c, &q.plan);
  if (!q.ev) cudaEventCreate(&q.ev);
  cudaEventRecord(q.ev, s->stream);
  q.state = 1;
  s->plainInflight.push_back(q.ticket);
  return vSuccess;
}

// mode 2: the request as one launch on its lane's stream, grid capped so
// that the lanes run side by side (continuous batching without a resident
// kernel: each admitted request starts at once on free SMs)
vResult_t launchLane(vserve* s, Request& q, int lane) {
  vcomm_t c = s->comms[q.nranks];
  cudaStream_t st = s->lanes[lane];
  if (!q.ev0) cudaEventCreate(&q.ev0);
  cudaEventRecord(q.ev0, st);
  vcommSetPlan(c, &q.plan);
  // FIFO protocols: requests of the same vrank count share comms[k] and its
  // FIFO arena, so they run one after another whatever lane they are on;
  // the direct protocol has no FIFO and needs no order
  const bool fifo = q.plan.proto != vProtoDirect;
  if (fifo && s->commEvUsed[q.nranks]) cudaStreamWaitEvent(st, s->commEv[q.nranks], 0);
  // a small lane's grid grows with the request (about 256 KiB of traffic per
  // CTA, 4..laneCtas CTAs): tiny requests stay on a few SMs, mid-size ones
  // are not starved
  int cap = s->laneCtas[lane];
  if (lane > 0) {
    const size_t bytes = (q.sb + q.rb) * (size_t)q.nranks;
    cap = (int)std::min<size_t>((size_t)cap, std::max<size_t>(4, bytes / (256u << 10)));
  }
  vResult_t r = serveCollective(q.coll, q.send, q.recv, q.count, q.dtype, q.redop, q.plan.proto, st, c,
                                cap, &q.plan);
  if (r != vSuccess) return r;
  if (fifo) {
    cudaEventRecord(s->commEv[q.nranks], st);
    s->commEvUsed[q.nranks] = true;
  }
  if (!q.ev) cudaEventCreate(&q.ev);
  cudaEventRecord(q.ev, st);
  q.state = 1;
  q.lane = lane;
  s->laneInflight[lane].push_back(q.ticket);
  return vSuccess;
}

// try to start the request at the head of `q` on gang g (-1: plain launch);
// false if the budget or the pool cannot take it yet
bool tryStart(vserve* s, std::deque<uint64_t>& q, int g) {
  Request& r = s->reqs[q.front()];
  const size_t bytes = (r.sb + r.rb) * r.nranks;
  if (s->inflight + bytes > s->cfg.memBudget) return false;
  if (s->cfg.mode == 3 && s->tileTicket[s->tilePosted % kTileRing]) return false;   // ring full
  if (!allocOutputs(s, r)) return false;
  s->inflight += bytes;
  s->maxInflight = std::max(s->maxInflight, s->inflight);
  if (s->cfg.mode == 3) {
    if (!postTile(s, r)) {   // the kernel could not be started
      s->threadErr = vCudaError;
      completeReq(s, r, false);
    }
  } else if (s->cfg.mode == 2) {
    vResult_t e = launchLane(s, r, g);
    if (e != vSuccess) {
      s->threadErr = e;
      completeReq(s, r, false);
    }
  } else if (g >= 0) {
    postToGang(s, r, g);
  } else {
    vResult_t e = launchPlain(s, r);
    if (e != vSuccess) {
      s->threadErr = e;
      completeReq(s, r, false);
    }
  }
  q.pop_front();
  return true;
}

void dispatcher(vserve* s) {
  cudaSetDevice(s->dev);
  while (!s->stop.load(std::memory_order_relaxed)) {
    bool progress = false;
    std::unique_lock<std::mutex> lk(s->mu);
    while (!s->incoming.empty()) {
      const uint64_t t = s->incoming.front();
      s->incoming.pop_front();
      (s->reqs[t].big ? s->bigQ : s->smallQ).push_back(t);
    }
    // completions
    if (s->cfg.mode == 0) {
      for (int g = 0; g < s->ngangs; g++) {
        if (!s->running[g]) continue;
        volatile ServeSlot* slot = &s->hSlots[g];
        const bool fin = slot->done >= s->posted[g];
        if (fin || slot->err) {
          Request& q = s->reqs[s->running[g]];
          if (fin) q.serviceNs = (int64_t)(slot->tEnd - slot->tStart);
          completeReq(s, q, fin && slot->err == 0);
          s->running[g] = 0;
          progress = true;
        }
      }
    } else if (s->cfg.mode == 3) {
      for (auto it = s->tileInflight.begin(); it != s->tileInflight.end();) {
        Request& q = s->reqs[*it];
        volatile TileDone* d = &s->hDone[q.gang];
        if (d->seq == q.tseq + 1) {
          q.serviceNs = (int64_t)(d->tEnd - d->tStart);
          s->tileTicket[q.gang] = 0;
          completeReq(s, q, true);
          it = s->tileInflight.erase(it);
          progress = true;
        } else {
          ++it;
        }
      }
      noteTilesExit(s);
      if (!s->tilesUp && s->hCtl->error) {
        // a bulk copy of the kernel timed out: what it did not finish has failed
        for (uint64_t t : s->tileInflight) {
          Request& q = s->reqs[t];
          s->tileTicket[q.gang] = 0;
          completeReq(s, q, false);
        }
        s->tileInflight.clear();
        s->threadErr = (vResult_t)s->hCtl->error;
      } else if (!s->tilesUp && !s->tileInflight.empty()) {
        // the kernel went idle just as requests were posted: the ones it did
        // not take (every one it took has completed) go to a new launch
        const uint64_t from = *(volatile unsigned long long*)&s->hCtl->ingested;
        bool pending = false;
        for (uint64_t t : s->tileInflight) pending = pending || s->reqs[t].tseq >= from;
        if (pending && launchTiles(s, from) != vSuccess) s->threadErr = vCudaError;
      }
    } else if (s->cfg.mode == 2) {
      for (size_t l = 0; l < s->lanes.size(); l++) {
        while (!s->laneInflight[l].empty()) {
          Request& q = s->reqs[s->laneInflight[l].front()];
          cudaError_t e = cudaEventQuery(q.ev);
          if (e == cudaErrorNotReady) break;
          (void)cudaGetLastError();
          vResult_t ae = vSuccess;
          vcommGetAsyncError(s->comms[q.nranks], &ae);
          float ms = 0;
          if (e == cudaSuccess && cudaEventElapsedTime(&ms, q.ev0, q.ev) == cudaSuccess)
            q.serviceNs = (int64_t)(ms * 1e6);
          (void)cudaGetLastError();
          completeReq(s, q, e == cudaSuccess && ae == vSuccess);
          s->laneInflight[l].pop_front();
          progress = true;
        }
      }
    } else {
      while (!s->plainInflight.empty()) {
        Request& q = s->reqs[s->plainInflight.front()];
        cudaError_t e = cudaEventQuery(q.ev);
        if (e == cudaErrorNotReady) break;
        (void)cudaGetLastError();
        vResult_t ae = vSuccess;
        vcommGetAsyncError(s->comms[q.nranks], &ae);
        float ms = 0;
        if (e == cudaSuccess && cudaEventElapsedTime(&ms, q.ev0, q.ev) == cudaSuccess)
          q.serviceNs = (int64_t)(ms * 1e6);
        (void)cudaGetLastError();
        completeReq(s, q, e == cudaSuccess && ae == vSuccess);
        s->plainInflight.pop_front();
        progress = true;
      }
    }
    // admission: first come first served within each size class; a class
    // whose head must wait (budget, pool, no free gang) does not hold up the other
    if (s->cfg.mode == 0) {
      while (!s->bigQ.empty() && !s->running[0] && tryStart(s, s->bigQ, 0)) progress = true;
      while (!s->smallQ.empty()) {
        int g = -1;
        for (int i = 1; i < s->ngangs && g < 0; i++)
          if (!s->running[i]) g = i;
        if (g < 0 && !s->running[0] && s->bigQ.empty()) g = 0;
        if (g < 0 || !tryStart(s, s->smallQ, g)) break;
        progress = true;
      }
    } else if (s->cfg.mode == 2) {
      // large requests on lane 0, the others on the least busy small lane;
      // at most two launches in flight per lane
      const size_t depth = 2;
      while (!s->bigQ.empty() && s->laneInflight[0].size() < depth && tryStart(s, s->bigQ, 0)) progress = true;
      while (!s->smallQ.empty()) {
        int best = -1;
        for (int l = 1; l < (int)s->lanes.size(); l++)
          if (s->laneInflight[l].size() < depth &&
              (best < 0 || s->laneInflight[l].size() < s->laneInflight[best].size()))
            best = l;
        if (best < 0 || !tryStart(s, s->smallQ, best)) break;
        progress = true;
      }
    } else {
      // one stream (mode 1) or the request ring (mode 3): requests start in
      // arrival order
      while (true) {
        std::deque<uint64_t>* q = nullptr;
        if (!s->bigQ.empty() && !s->smallQ.empty())
          q = (s->reqs[s->bigQ.front()].arrivalNs <= s->reqs[s->smallQ.front()].arrivalNs) ? &s->bigQ : &s->smallQ;
        else if (!s->bigQ.empty()) q = &s->bigQ;
        else if (!s->smallQ.empty()) q = &s->smallQ;
        if (!q || !tryStart(s, *q, -1)) break;
        progress = true;
      }
    }
    lk.unlock();
    if (!progress) std::this_thread::yield();
  }
}

}  // namespace

extern "C" {

vResult_t vServeCreate(vserve_t* out, const vserveConfig_t* cfgIn) {
  if (!out) return vInvalidArgument;
  *out = nullptr;
  vserveConfig_t cfg{};
  if (cfgIn) cfg = *cfgIn;
  if (cfg.maxRanks <= 0) cfg.maxRanks = kServeMaxRanks;
  if (cfg.memBudget == 0) cfg.memBudget = (size_t)40 << 30;
  if (cfg.threads <= 0) cfg.threads = 512;
  if (cfg.smallGangs < 0) cfg.smallGangs = 0;
  if (cfg.smallGangs == 0 && !(cfgIn && cfgIn->smallGangs == 0)) cfg.smallGangs = 1;
  if (cfg.bigThreshold == 0) cfg.bigThreshold = (size_t)4 << 20;
  const size_t defSlot[3] = {256u << 10, 32u << 10, 300u << 10};
  for (int p = 0; p < 3; p++)
    if (cfg.slotBytes[p] == 0) cfg.slotBytes[p] = defSlot[p];
  if (cfg.idleTimeoutSec <= 0) cfg.idleTimeoutSec = 30.0;
  if (cfg.mode < 0 || cfg.mode > 3 || cfg.maxRanks > kServeMaxRanks ||
      1 + cfg.smallGangs > kMaxServeGangs || cfg.threads % 64 || cfg.threads > 512)
    return vInvalidArgument;
  for (int p = 0; p < 3; p++)
    if (cfg.slotBytes[p] % 256) return vInvalidArgument;

  vserve* s = new vserve();
  s->cfg = cfg;
  vResult_t r = fromCudaS(cudaGetDevice(&s->dev));
  if (r == vSuccess) r = fromCudaS(cudaDeviceGetAttribute(&s->nsm, cudaDevAttrMultiProcessorCount, s->dev));
  if (r == vSuccess) r = fromCudaS(cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking));
  if (r == vSuccess) r = fromCudaS(cudaMalloc(&s->pool, cfg.memBudget));
  if (r == vSuccess) s->alloc.init(cfg.memBudget);
  const int kmax = cfg.maxRanks;
  if (r == vSuccess && cfg.mode == 0) {
    int per = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, serveKernel(), cfg.threads, 0) != cudaSuccess) {
      (void)cudaGetLastError();
      per = 0;
    }
    // by default the wide gang takes every co-resident CTA the narrow ones leave
    if (cfg.bigGangChannels <= 0)
      cfg.bigGangChannels = std::max(1, (per * s->nsm - cfg.smallGangs * kmax) / kmax);
    s->cfg.bigGangChannels = cfg.bigGangChannels;
    s->ngangs = 1 + cfg.smallGangs;
    s->gangCpg.assign(s->ngangs, 1);
    s->gangCpg[0] = cfg.bigGangChannels;
    int totalCh = 0;
    for (int c : s->gangCpg) totalCh += c;
    const int ctas = totalCh * kmax;
    if ((long long)per * s->nsm < ctas) r = vUnsupported;   // gangs must be co-resident
    // mailboxes, error and shutdown words (host-mapped), gang state (device)
    if (r == vSuccess) r = fromCudaS(cudaHostAlloc((void**)&s->hSlots, sizeof(ServeSlot) * s->ngangs, cudaHostAllocMapped));
    if (r == vSuccess) r = fromCudaS(cudaHostGetDevicePointer((void**)&s->dSlots, s->hSlots, 0));
    if (r == vSuccess) memset(s->hSlots, 0, sizeof(ServeSlot) * s->ngangs);
    if (r == vSuccess) r = fromCudaS(cudaHostAlloc((void**)&s->hShutdown, sizeof(int), cudaHostAllocMapped));
    if (r == vSuccess) r = fromCudaS(cudaHostGetDevicePointer((void**)&s->dShutdown, s->hShutdown, 0));
    if (r == vSuccess) r = fromCudaS(cudaHostAlloc((void**)&s->hErr, sizeof(ErrWord), cudaHostAllocMapped));
    if (r == vSuccess) r = fromCudaS(cudaHostGetDevicePointer((void**)&s->dErr, s->hErr, 0));
    if (r == vSuccess) r = fromCudaS(cudaHostAlloc((void**)&s->hAbort, sizeof(int), cudaHostAllocMapped));
    if (r == vSuccess) r = fromCudaS(cudaHostGetDevicePointer((void**)&s->dAbort, s->hAbort, 0));
    if (r == vSuccess) {
      *(volatile int*)s->hShutdown = 0;
      *(volatile int*)s->hAbort = 0;
      memset(s->hErr, 0, sizeof(ErrWord));
    }
    if (r == vSuccess) r = fromCudaS(cudaMalloc(&s->dGangs, sizeof(ServeGang) * s->ngangs));
    if (r == vSuccess) r = fromCudaS(cudaMemset(s->dGangs, 0, sizeof(ServeGang) * s->ngangs));
    if (r == vSuccess) r = fromCudaS(cudaMalloc(&s->dClaim, sizeof(int)));
    if (r == vSuccess) r = fromCudaS(cudaMemset(s->dClaim, 0, sizeof(int)));
    // ring arenas, one per protocol, for all gangs' channels
    const int nconn = totalCh * kmax;
    for (int p = 0; p < 3 && r == vSuccess; p++) {
      const size_t bytes = (size_t)nconn * 8 * cfg.slotBytes[p];
      r = fromCudaS(cudaMalloc(&s->arenaBuf[p], bytes));
      if (r == vSuccess) r = fromCudaS(cudaMemset(s->arenaBuf[p], 0, bytes));
      const size_t ctrB = (size_t)nconn * 2 * kCounterStride * 8;
      if (r == vSuccess) r = fromCudaS(cudaMalloc(&s->arenaCtr[p], ctrB));
      if (r == vSuccess) r = fromCudaS(cudaMemset(s->arenaCtr[p], 0, ctrB));
      std::vector<ConnDev> h(nconn);
      for (int i = 0; i < nconn; i++) {
        h[i].buf = s->arenaBuf[p] + (size_t)i * 8 * cfg.slotBytes[p];
        h[i].tail = s->arenaCtr[p] + (size_t)(2 * i) * kCounterStride;
        h[i].head = s->arenaCtr[p] + (size_t)(2 * i + 1) * kCounterStride;
        h[i].unused = 0;
      }
      if (r == vSuccess) r = fromCudaS(cudaMalloc(&s->arenaConns[p], nconn * sizeof(ConnDev)));
      if (r == vSuccess)
        r = fromCudaS(cudaMemcpy(s->arenaConns[p], h.data(), nconn * sizeof(ConnDev), cudaMemcpyHostToDevice));
    }
    if (r == vSuccess) r = fromCudaS(cudaDeviceSynchronize());
    if (r == vSuccess) {
      ServeArgs a;
      memset(&a, 0, sizeof(a));
      a.slots = s->dSlots;
      a.gangs = s->dGangs;
      a.shutdown = s->dShutdown;
      a.errClaim = s->dClaim;
      a.err = s->dErr;
      a.abortFlag = s->dAbort;
      a.timeoutNs = 5000000000ull;
      a.idleTimeoutNs = (unsigned long long)(cfg.idleTimeoutSec * 1e9);
      for (int p = 0; p < 3; p++) a.conns[p] = s->arenaConns[p];
      a.ngangs = s->ngangs;
      a.kmax = kmax;
      a.nsteps = 8;
      int cta = 0, conn = 0;
      for (int g = 0; g < s->ngangs; g++) {
        a.gangCta[g] = cta;
        a.gangCpg[g] = s->gangCpg[g];
        a.gangConn[g] = conn;
        cta += s->gangCpg[g] * kmax;
        conn += s->gangCpg[g] * kmax;
      }
      a.gangCta[s->ngangs] = cta;
      void* args[] = {(void*)&a};
      r = fromCudaS(cudaLaunchCooperativeKernel(serveKernel(), dim3(cta), dim3(cfg.threads), args,
                                                0, s->stream));
      if (r == vSuccess) s->kernelUp = true;
    }
    s->posted.assign(s->ngangs, 0);
    s->running.assign(s->ngangs, 0);
  }
  if (r == vSuccess && cfg.mode == 2) {
    // one stream per lane; small lanes get a few SMs each, the large lane the rest
    const int nSmall = std::max(1, cfg.smallGangs);
    const int reserve = 16;   // SMs the large lane leaves to the small lanes
    s->lanes.assign(1 + nSmall, nullptr);
    s->laneCtas.assign(1 + nSmall, 32);
    s->laneCtas[0] = std::max(4, s->nsm - reserve);
    s->laneInflight.assign(1 + nSmall, std::deque<uint64_t>());
    for (auto& st : s->lanes)
      if (r == vSuccess) r = fromCudaS(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    for (int k = 0; k <= kServeMaxRanks && r == vSuccess; k++)
      r = fromCudaS(cudaEventCreateWithFlags(&s->commEv[k], cudaEventDisableTiming));
  }
  if (r == vSuccess && cfg.mode == 3) {
    // the pipeline stages take the shared memory the kernel's own leaves
    int maxSmem = 0;
    cudaFuncAttributes fa{};
    r = fromCudaS(cudaDeviceGetAttribute(&maxSmem, cudaDevAttrMaxSharedMemoryPerBlockOptin, s->dev));
    if (r == vSuccess) r = fromCudaS(cudaFuncGetAttributes(&fa, serveTilesKernel()));
    if (r == vSuccess) {
      const long long room = (long long)maxSmem - (long long)fa.sharedSizeBytes - (long long)serveTilesSmem(0);
      s->tileStageBytes = room > 0 ? (unsigned)(room / serveTilesStages() / 128 * 128) : 0;
      if (s->tileStageBytes < 16 * 128) r = vUnsupported;   // a 128-byte sub-tile for each of 16 inputs
    }
    if (r == vSuccess)
      r = fromCudaS(cudaFuncSetAttribute(serveTilesKernel(), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)serveTilesSmem(s->tileStageBytes)));
    int per = 0;
    if (r == vSuccess &&
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, serveTilesKernel(), serveTilesThreads(),
                                                      serveTilesSmem(s->tileStageBytes)) != cudaSuccess) {
      (void)cudaGetLastError();
      per = 0;
    }
    s->tileWorkers = per * s->nsm - 1;   // CTA 0 ingests
    if (r == vSuccess && s->tileWorkers < 1) r = vUnsupported;
    if (r == vSuccess) r = fromCudaS(cudaHostAlloc((void**)&s->hRing, sizeof(TileReq) * kTileRing, cudaHostAllocMapped));
    if (r == vSuccess) r = fromCudaS(cudaHostGetDevicePointer((void**)&s->dRing, s->hRing, 0));
    if (r == vSuccess) memset(s->hRing, 0, sizeof(TileReq) * kTileRing);
    if (r == vSuccess) r = fromCudaS(cudaHostAlloc((void**)&s->hDone, sizeof(TileDone) * kTileRing, cudaHostAllocMapped));
    if (r == vSuccess) r = fromCudaS(cudaHostGetDevicePointer((void**)&s->dDone, s->hDone, 0));
    if (r == vSuccess) memset(s->hDone, 0, sizeof(TileDone) * kTileRing);
    if (r == vSuccess) r = fromCudaS(cudaHostAlloc((void**)&s->hCtl, sizeof(TileCtl), cudaHostAllocMapped));
    if (r == vSuccess) r = fromCudaS(cudaHostGetDevicePointer((void**)&s->dCtl, s->hCtl, 0));
    if (r == vSuccess) memset(s->hCtl, 0, sizeof(TileCtl));
    if (r == vSuccess) r = fromCudaS(cudaMalloc(&s->dState, sizeof(TileState) * kTileRing));
    if (r == vSuccess) r = fromCudaS(cudaMemset(s->dState, 0, sizeof(TileState) * kTileRing));
    if (r == vSuccess) r = fromCudaS(cudaMalloc(&s->dQueues, sizeof(TileQueues)));
    if (r == vSuccess) r = fromCudaS(cudaMemset(s->dQueues, 0, sizeof(TileQueues)));
    if (r == vSuccess) r = fromCudaS(cudaEventCreateWithFlags(&s->tilesEnd, cudaEventDisableTiming));
    if (r == vSuccess) r = fromCudaS(cudaDeviceSynchronize());
    s->tileTicket.assign(kTileRing, 0);
    if (r == vSuccess) r = launchTiles(s, 0);
  }
  if (r == vSuccess && (cfg.mode == 1 || cfg.mode == 2)) {
    // one communicator per vrank count, arenas allocated now (not mid-stream)
    vcommConfig_t cc{};
    for (int p = 0; p < 3; p++) cc.slotBytes[p] = cfg.slotBytes[p];
    for (int k = 1; k <= kmax && r == vSuccess; k++) {
      r = vcommInitConfig(&s->comms[k], k, std::min(VCOMM_MAX_CHANNELS, std::max(1, 2 * s->nsm / k)), &cc);
      if (r == vSuccess && k > 1) r = vcommPrepare(s->comms[k], 1u << vAlgoRing, 0xEu);
    }
  }
  if (r == vSuccess && cfg.mode >= 1) preloadKernels(cfg.mode);
  if (r != vSuccess) {
    vServeDestroy(s);
    return r;
  }
  s->th = std::thread(dispatcher, s);
  *out = s;
  return vSuccess;
}

vResult_t vServeSubmit(vserve_t s, int coll, const void* const* sendbufs, size_t count,
                       vDataType_t dtype, vRedOp_t op, int nranks, vProto_t proto, int flags,
                       int64_t arrivalNs, uint64_t* ticket) {
  if (!s || !sendbufs || !ticket || count == 0) return vInvalidArgument;
  if (coll != kAllReduce && coll != kReduceScatter && coll != kAllGather) return vUnsupported;
  if (nranks < 1 || nranks > s->cfg.maxRanks || dtype < vInt32 || dtype > vBfloat16 ||
      op < vSum || op > vMax || proto < vProtoAuto || proto > vProtoDirect)
    return vInvalidArgument;
  Request q;
  q.coll = coll;
  q.dtype = dtype;
  q.redop = op;
  q.nranks = nranks;
  q.flags = flags;
  // gangs have no cluster protocol; the tile kernel runs the direct protocol only
  q.proto = (proto == vProtoCluster) ? vProtoLL : proto;
  if (s->cfg.mode == 3 && proto != vProtoAuto && proto != vProtoDirect) return vUnsupported;
  q.count = count;
  const size_t esz = (dtype == vFloat16 || dtype == vBfloat16) ? 2 : 4;
  q.sb = count * esz;
  q.rb = count * esz;
  if (coll == kReduceScatter) q.sb = (size_t)nranks * count * esz;
  if (coll == kAllGather) q.rb = (size_t)nranks * count * esz;
  if ((q.sb + q.rb) * nranks > s->cfg.memBudget) return vInvalidArgument;   // could never be admitted
  for (int r = 0; r < nranks; r++) {
    if (!sendbufs[r] || (uintptr_t)sendbufs[r] % esz) return vInvalidArgument;
    q.send[r] = sendbufs[r];
  }
  q.arrivalNs = arrivalNs ? arrivalNs : nowNs();
  planFor(s, q);
  std::lock_guard<std::mutex> lk(s->mu);
  q.ticket = s->nextTicket++;
  *ticket = q.ticket;
  s->reqs.emplace(q.ticket, q);
  s->incoming.push_back(q.ticket);
  s->submitted++;
  return vSuccess;
}

vResult_t vServeQuery(vserve_t s, uint64_t ticket, int* state, int64_t* latencyNs,
                      int64_t* serviceNs, vPlan_t* plan, void** recvbufs) {
  if (!s || !state) return vInvalidArgument;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return vInvalidArgument;
  const Request& q = it->second;
  *state = q.state;
  if (latencyNs) *latencyNs = q.state >= 2 ? q.doneNs - q.arrivalNs : -1;
  if (serviceNs) *serviceNs = q.serviceNs;
  if (plan) *plan = q.plan;
  if (recvbufs)
    for (int r = 0; r < q.nranks; r++) recvbufs[r] = q.recv[r];
  return vSuccess;
}

vResult_t vServeRelease(vserve_t s, uint64_t ticket) {
  if (!s) return vInvalidArgument;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end() || it->second.state < 2) return vInvalidArgument;
  Request& q = it->second;
  if (!(q.flags & 1)) {
    for (int r = 0; r < q.nranks; r++)
      if (q.recv[r]) s->alloc.release(q.poolOff[r], q.rb);
    s->inflight -= (q.sb + q.rb) * q.nranks;
  }
  if (q.ev) cudaEventDestroy(q.ev);
  if (q.ev0) cudaEventDestroy(q.ev0);
  s->reqs.erase(it);
  return vSuccess;
}

vResult_t vServeGetStats(vserve_t s, vserveStats_t* st) {
  if (!s || !st) return vInvalidArgument;
  std::lock_guard<std::mutex> lk(s->mu);
  st->submitted = s->submitted;
  st->completed = s->completed;
  st->failed = s->failed;
  st->inflightBytes = s->inflight;
  st->maxInflightBytes = s->maxInflight;
  st->queued = s->bigQ.size() + s->smallQ.size() + s->incoming.size();
  return s->threadErr;
}

vResult_t vServeDestroy(vserve_t s) {
  if (!s) return vSuccess;
  s->stop.store(true);
  if (s->th.joinable()) s->th.join();
  if (s->hShutdown) *(volatile int*)s->hShutdown = 1;
  if (s->hCtl) *(volatile int*)&s->hCtl->shutdown = 1;   // the tile kernel drains, then returns
  if (s->stream) cudaStreamSynchronize(s->stream);
  for (auto st : s->lanes)
    if (st) cudaStreamSynchronize(st);
  for (auto& kv : s->reqs) {
    if (kv.second.ev) cudaEventDestroy(kv.second.ev);
    if (kv.second.ev0) cudaEventDestroy(kv.second.ev0);
  }
  for (int k = 0; k <= kServeMaxRanks; k++)
    if (s->commEv[k]) cudaEventDestroy(s->commEv[k]);
  for (int k = 0; k <= kServeMaxRanks; k++)
    if (s->comms[k]) vcommDestroy(s->comms[k]);
  for (int p = 0; p < 3; p++) {
    if (s->arenaBuf[p]) cudaFree(s->arenaBuf[p]);
    if (s->arenaCtr[p]) cudaFree(s->arenaCtr[p]);
    if (s->arenaConns[p]) cudaFree(s->arenaConns[p]);
  }
  if (s->hRing) cudaFreeHost(s->hRing);
  if (s->hDone) cudaFreeHost(s->hDone);
  if (s->hCtl) cudaFreeHost(s->hCtl);
  if (s->dState) cudaFree(s->dState);
  if (s->dQueues) cudaFree(s->dQueues);
  if (s->tilesEnd) cudaEventDestroy(s->tilesEnd);
  if (s->dGangs) cudaFree(s->dGangs);
  if (s->dClaim) cudaFree(s->dClaim);
  if (s->hSlots) cudaFreeHost(s->hSlots);
  if (s->hShutdown) cudaFreeHost(s->hShutdown);
  if (s->hErr) cudaFreeHost(s->hErr);
  if (s->hAbort) cudaFreeHost(s->hAbort);
  if (s->pool) cudaFree(s->pool);
  if (s->stream) cudaStreamDestroy(s->stream);
  for (auto st : s->lanes)
    if (st) cudaStreamDestroy(st);
  (void)cudaGetLastError();
  delete s;
  return vSuccess;
}

}  // extern "C"
