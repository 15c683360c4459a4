// vcomm_serve_tiles.cu -- serving mode 3: direct-protocol requests as tiles
// of one resident kernel.
//
// The host appends requests to a ring in host-mapped memory.  CTA 0 of the
// kernel (one warp) ingests them in order: it copies each entry into device
// state and publishes it on one of two device queues, small requests and
// large ones.  Every other CTA takes the next tile of the first request of
// the small queue that still has tiles, else of the large queue, and folds
// its 16-byte units exactly as the direct protocol's kernels do (each unit's
// ring chain in the ring schedule's order, so the bits are those of a
// per-call launch with the same plan).  The CTA that finishes a request's
// last tile writes its completion into host-mapped memory.  A small request
// that arrives while a large one runs takes the next free CTAs, so it waits
// for a tile at most, never for the large request; large requests share the
// GPU tile by tile in arrival order.
//
// Data movement.  A tile of a 16-byte aligned request is a byte range of one
// block (AllReduce: the buffer; ReduceScatter / AllGather: block b) that moves
// through shared memory in sub-tiles: thread 0 issues bulk asynchronous copies
// of the sub-tile's inputs (k for a reduction, one for AllGather) into one of
// three stages, all threads fold the stage into an output buffer, and thread 0
// bulk-stores it to every output.  The stages run ahead across tile
// boundaries (thread 0 claims the next tile while the current one is still
// folding), so the loads in flight never drain between tiles.  Unaligned
// requests take the register kernels' element-wise path, one tile at a time.
//
// No CTA waits on another: claims and completions are atomics, and the only
// waits are the idle polls (bounded by the idle timeout and the stop word)
// and the waits for this CTA's own bulk copies (bounded by copyTimeoutNs).
#include <cuda_runtime.h>

#include <cstddef>

#include "vcomm_direct.cuh"
#include "vcomm_kernels.h"

namespace vc {
namespace {

using namespace direct;

constexpr int kTileThreads = 256;
constexpr int kTileStages = 3;
constexpr unsigned kTileOutBytes = 16384;   // one folded sub-tile, double buffered
constexpr int kTileNU = 2;                  // register path: units per thread per iteration

VDEV uint64_t ldAcquireSys(const unsigned long long* p) {
  uint64_t v;
  asm volatile("ld.acquire.sys.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
VDEV uint64_t ldVol(const unsigned long long* p) { return *(const volatile unsigned long long*)p; }
VDEV void stVol(unsigned long long* p, uint64_t v) { *(volatile unsigned long long*)p = v; }
// every store group but the newest kDoneLag has completed (its global writes)
constexpr int kDoneLag = 4;
VDEV void bulkWaitDoneLag() { asm volatile("cp.async.bulk.wait_group 4;" ::: "memory"); }
// the completed bulk stores' global writes, ordered before what follows
VDEV void fenceProxyGlobal() { asm volatile("fence.proxy.async.global;" ::: "memory"); }

VDEV DirectView viewOfReq(const ServeReq* q) {
  return DirectView{(const void* const*)q->send, (void* const*)q->recv, q->count, q->chunk, q->inplaceMask,
                    q->coll, q->nranks, q->nsub, q->root, 0};
}

// ---- register path (requests that are not 16-byte aligned; vec 2: aligned
// buffers whose blocks are not whole 16-byte units), one body per (dtype,
// op), out of line
template <class T, class Op>
__device__ __noinline__ void tileReduce(const ServeReq* q, unsigned long long lo, unsigned long long hi,
                                        bool tail) {
  const DirectView v = viewOfReq(q);
  if (q->vec == 1) directReduce<T, Op, Unit16L2<T>, kTileNU>(v, lo, hi, tail);
  else if (q->vec == 2) directReduceShifted<T, Op, L2Mem, kTileNU>(v, lo, hi, tail);
  else directReduce<T, Op, Unit1L2<T>, 1>(v, lo, hi, tail);
}

__device__ __noinline__ void tileCopy(const ServeReq* q, unsigned long long lo, unsigned long long hi, bool tail) {
  const DirectView v = viewOfReq(q);
  if (q->vec == 1) directCopy<Unit16L2<uint8_t>>(v, lo, hi, tail);
  else if (q->vec == 2) directCopyShifted<L2Mem>(v, lo, hi, tail);
  else directCopy<Unit1L2<uint8_t>>(v, lo, hi, tail);
}

__device__ void runTile(const ServeReq* q, unsigned long long lo, unsigned long long hi, bool tail) {
  if (q->coll == kAllGather || q->coll == kBroadcast) {
    tileCopy(q, lo, hi, tail);
    return;
  }
  const bool mx = q->redop == kMax;
  if (q->dtype == kI32) mx ? tileReduce<int32_t, OpMax>(q, lo, hi, tail) : tileReduce<int32_t, OpSum>(q, lo, hi, tail);
  else if (q->dtype == kF32) mx ? tileReduce<float, OpMax>(q, lo, hi, tail) : tileReduce<float, OpSum>(q, lo, hi, tail);
  else if (q->dtype == kF16) mx ? tileReduce<__half, OpMax>(q, lo, hi, tail) : tileReduce<__half, OpSum>(q, lo, hi, tail);
  else mx ? tileReduce<__nv_bfloat16, OpMax>(q, lo, hi, tail) : tileReduce<__nv_bfloat16, OpSum>(q, lo, hi, tail);
}

// ---- staged path: fold one sub-tile of `len` bytes from the stage at
// shared-memory byte offset `in` (inputs `sub` bytes apart) into the output
// buffer at offset `o` (offsets into the kernel's dynamic shared memory, read
// through the array itself so the loads are ordinary shared loads).  Unit
// u's chain starts at rank seg[i] + 1 for the first i with u < segEnd[i]
// (thread 0 has cut the sub-tile into its ring segments); a unit's k inputs
// are loaded before they are folded.
constexpr int kMaxSegRuns = 4;

template <class T, class Op>
__device__ __noinline__ void foldStage(const ServeReq* q, unsigned in, unsigned sub, unsigned o, unsigned len,
                                       unsigned long long off, const int* seg, const unsigned* segEnd, int nseg) {
  extern __shared__ __align__(128) unsigned char smem[];
  const int k = q->nranks;
  unsigned long long runEnd = 0;   // nseg == 0: each unit's segment from the partition
  int s0 = 0;
  for (unsigned u = threadIdx.x * 16u; u < len; u += blockDim.x * 16u) {
    int s;
    if (nseg > 0) {
      int i = 0;
      while (i + 1 < nseg && u >= segEnd[i]) i++;
      s = seg[i];
    } else {
      const unsigned long long e0 = (off + u) / sizeof(T);
      if (e0 >= runEnd) s0 = arSegment(viewOfReq(q), e0, (int)sizeof(T), &runEnd);
      s = s0;
    }
    int r = s + 1 < k ? s + 1 : 0;
    uint4 x[kServeMaxRanks];
#pragma unroll
    for (int j = 0; j < kServeMaxRanks; j++) {
      if (j < k) {
        x[j] = *(const uint4*)(smem + in + (unsigned)r * sub + u);
        if (++r == k) r = 0;
      }
    }
    uint4 acc = x[0];
#pragma unroll
    for (int j = 1; j < kServeMaxRanks; j++)
      if (j < k) acc = combine<T, Op, uint4>(acc, x[j]);
    *(uint4*)(smem + o + u) = acc;
  }
}

__device__ __noinline__ void copyStage(unsigned in, unsigned o, unsigned len) {
  extern __shared__ __align__(128) unsigned char smem[];
  for (unsigned u = threadIdx.x * 16u; u < len; u += blockDim.x * 16u)
    *(uint4*)(smem + o + u) = *(const uint4*)(smem + in + u);
}

VDEV void foldStageAny(const ServeReq* q, unsigned in, unsigned sub, unsigned o, unsigned len,
                       unsigned long long off, const int* seg, const unsigned* segEnd, int nseg) {
  if (q->coll == kAllGather) {   // a copy: the one input as it is
    copyStage(in, o, len);
    return;
  }
  const bool mx = q->redop == kMax;
#define VC_FOLD(T) mx ? foldStage<T, OpMax>(q, in, sub, o, len, off, seg, segEnd, nseg) \
                      : foldStage<T, OpSum>(q, in, sub, o, len, off, seg, segEnd, nseg)
  if (q->dtype == kI32) VC_FOLD(int32_t);
  else if (q->dtype == kF32) VC_FOLD(float);
  else if (q->dtype == kF16) VC_FOLD(__half);
  else VC_FOLD(__nv_bfloat16);
#undef VC_FOLD
}

// thread 0: the ring segments of a sub-tile (bytes [off, off + len) of block
// b): AllReduce segments from the partition (a segment is normally a chunk,
// far longer than a sub-tile; 0 runs if the sub-tile holds more than
// kMaxSegRuns, as the short segments of a small buffer's last loop do, and
// the fold then looks each unit's segment up); ReduceScatter block b is one run
VDEV int cutSegments(const ServeReq* q, int b, unsigned long long off, unsigned len, int* seg, unsigned* segEnd) {
  if (q->coll != kAllReduce) {
    seg[0] = b;
    segEnd[0] = len;
    return 1;
  }
  const DirectView v = viewOfReq(q);
  const unsigned long long esz = (q->dtype == kF16 || q->dtype == kBF16) ? 2 : 4;
  unsigned u = 0;
  int n = 0;
  while (u < len) {
    if (n == kMaxSegRuns) return 0;
    unsigned long long runEnd;   // in elements
    seg[n] = arSegment(v, (off + u) / esz, (int)esz, &runEnd);
    const unsigned long long endB = runEnd * esz - off;
    segEnd[n] = endB < len ? (unsigned)endB : len;
    u = segEnd[n];
    n++;
  }
  return n;
}

// the element tail of a staged AllReduce (count not a multiple of the units)
template <class T, class Op>
__device__ __noinline__ void tailReduce(const ServeReq* q) {
  const DirectView v = viewOfReq(q);
  constexpr unsigned long long E = 16 / sizeof(T);
  const unsigned long long nunit = q->count / E;
  const unsigned long long nt = q->count - nunit * E;
  for (unsigned long long t = threadIdx.x; t < nt; t += blockDim.x) {
    const unsigned long long i = nunit * E + t;
    unsigned long long re;
    const int s = arSegment(v, i, (int)sizeof(T), &re);
    const T x = foldChain<T, Op, Unit1L2<T>>(v, s, i * sizeof(T));
    for (int r = 0; r < q->nranks; r++) *(T*)((char*)v.recv[r] + i * sizeof(T)) = x;
  }
}

VDEV void tailAny(const ServeReq* q) {
  const bool mx = q->redop == kMax;
  if (q->dtype == kI32) mx ? tailReduce<int32_t, OpMax>(q) : tailReduce<int32_t, OpSum>(q);
  else if (q->dtype == kF32) mx ? tailReduce<float, OpMax>(q) : tailReduce<float, OpSum>(q);
  else if (q->dtype == kF16) mx ? tailReduce<__half, OpMax>(q) : tailReduce<__half, OpSum>(q);
  else mx ? tailReduce<__nv_bfloat16, OpMax>(q) : tailReduce<__nv_bfloat16, OpSum>(q);
}

VDEV bool hasTail(const ServeReq* q) {
  if (q->coll != kAllReduce) return false;
  const unsigned long long E = (q->dtype == kF16 || q->dtype == kBF16) ? 8 : 4;
  return q->count % E != 0;
}

// ---- CTA 0, warp 0: ingest ring entries firstSeq, firstSeq + 1, ... in order
__device__ void ingest(const TileArgs& a) {
  const int lane = threadIdx.x & 31;
  TileQueues* q = a.q;
  volatile TileCtl* ctl = a.ctl;
  unsigned long long next = a.firstSeq;
  uint64_t idle0 = globaltimer(), drain0 = 0;
  constexpr int kWords = (int)(offsetof(TileReq, seq) / 8);   // req .. klass
  static_assert(offsetof(TileReq, seq) == offsetof(TileState, next), "TileReq / TileState layouts differ");
  while (true) {
    int stop = 0, got = 0;
    if (lane == 0) {
      if (*(volatile int*)&q->stop) {
        stop = 1;   // a worker failed
      } else if (ctl->shutdown) {
        // stop taking requests; stop once every ingested one has completed
        const uint64_t now = globaltimer();
        if (drain0 == 0) drain0 = now;
        if (ldVol(&q->completed) >= next || now - drain0 > a.drainTimeoutNs) stop = 1;
      } else {
        TileReq* r = &a.ring[next % kTileRing];
        if (ldAcquireSys(&r->seq) == next + 1) {
          got = 1;
        } else if (globaltimer() - idle0 > a.idleTimeoutNs && ldVol(&q->completed) >= next) {
          stop = 1;   // idle: nothing posted for the idle timeout and nothing in progress
        }
      }
    }
    stop = __shfl_sync(0xffffffffu, stop, 0);
    got = __shfl_sync(0xffffffffu, got, 0);
    if (stop) break;
    if (!got) {
      __nanosleep(256);
      continue;
    }
    const int slot = (int)(next % kTileRing);
    const volatile unsigned long long* src = (const volatile unsigned long long*)&a.ring[slot];
    unsigned long long* dst = (unsigned long long*)&a.state[slot];
    for (int i = lane; i < kWords; i += 32) dst[i] = src[i];
    __syncwarp();
    if (lane == 0) {
      TileState* st = &a.state[slot];
      st->next = 0;
      st->done = 0;
      st->seq = next + 1;
      st->tStart = globaltimer();
      const int c = st->klass ? 1 : 0;
      __threadfence();                                   // the state before its queue entry
      const unsigned long long pos = q->tail[c];         // this warp is the only writer
      stVol(&q->entry[c][pos % kTileRing], (pos << 32) | (unsigned long long)(slot + 1));
      __threadfence();
      stRelease(&q->tail[c], pos + 1);
      stVol((unsigned long long*)&ctl->ingested, next + 1);
    }
    __syncwarp();
    next++;
    idle0 = globaltimer();
  }
  if (lane == 0) {
    __threadfence();
    atomicExch(&q->stop, 1);
    ctl->stopped = 1;
    __threadfence_system();
  }
}

// ---- where tiles come from.  The engine below calls a source from thread 0:
//   claim(&tile)        the next tile: an op id (>= 0) and its tile index; -1: none now
//   loadReq(id, dst)    the op's description, into shared memory
//   geom(id, tile, &w)  the tile's work: a byte range of one block (staged),
//                       or a range of the register kernels' units
//   done(id)            a tile of op `id` has completed (its stores are visible)
//   finished()          no tile will come any more
//   fail()              a bulk copy did not complete in time
struct TileWork {
  int staged, b, tail;                  // staged: block b; tail: also the element tail
  unsigned long long off, end;          // staged: bytes [off, end) of block b
  unsigned long long lo, hi;            // register path: units [lo, hi)
};

VDEV void stagedGeom(unsigned long long tile, unsigned long long perBlock, unsigned long long tileBytes,
                     unsigned long long blockBytes, unsigned long long ntiles, TileWork* w) {
  w->staged = 1;
  w->b = (int)(tile / perBlock);
  w->off = (tile % perBlock) * tileBytes;
  w->end = w->off + tileBytes < blockBytes ? w->off + tileBytes : blockBytes;
  w->tail = (tile + 1 == ntiles) ? 1 : 0;   // the request's element tail, if it has one
}
VDEV void registerGeom(unsigned long long tile, unsigned long long tileUnits, unsigned long long units,
                       unsigned long long ntiles, TileWork* w) {
  w->staged = 0;
  w->lo = tile * tileUnits;
  w->hi = w->lo + tileUnits < units ? w->lo + tileUnits : units;
  if (w->lo > w->hi) w->lo = w->hi;
  w->tail = (tile + 1 == ntiles) ? 1 : 0;
}

// the serving queues (small requests first), claimed with atomics
struct ServeSource {
  const TileArgs& a;
  VDEV long long claim(unsigned long long* tile) {
    TileQueues* q = a.q;
    for (int c = 0; c < 2; c++) {
      unsigned long long h = ldVol(&q->head[c]);
      const unsigned long long t = ldAcquire(&q->tail[c]);
      while (h < t) {
        const unsigned long long e = ldVol(&q->entry[c][h % kTileRing]);
        if ((e >> 32) != (h & 0xffffffffull)) break;   // not this position (cannot happen after tail)
        const int s = (int)(e & 0xffffffffull) - 1;
        TileState* st = &a.state[s];
        const unsigned long long tl = atomicAdd(&st->next, 1ull);
        if (tl < ldVol(&st->ntiles)) {
          *tile = tl;
          return s;
        }
        atomicCAS(&q->head[c], h, h + 1);               // every tile of entry h is claimed
        h++;
      }
    }
    return -1;
  }
  VDEV void loadReq(long long id, ServeReq* dst) {
    const unsigned long long* src = (const unsigned long long*)&a.state[id].req;
    for (int i = 0; i < (int)(sizeof(ServeReq) / 8); i++) ((unsigned long long*)dst)[i] = ldVol(&src[i]);
  }
  VDEV void geom(long long id, unsigned long long tile, TileWork* w) {
    TileState* st = &a.state[id];
    if (ldVol(&st->staged))
      stagedGeom(tile, ldVol(&st->perBlock), ldVol(&st->tileBytes), ldVol(&st->blockBytes), ldVol(&st->ntiles), w);
    else
      registerGeom(tile, ldVol(&st->tileUnits), ldVol(&st->units), ldVol(&st->ntiles), w);
  }
  // the CTA that finishes a request's last tile reports the request
  VDEV void done(long long id) {
    TileState* st = &a.state[id];
    fenceProxyGlobal();
    __threadfence();                                     // the tile's stores before the count
    const unsigned long long d = atomicAdd(&st->done, 1ull);
    if (d + 1 == ldVol(&st->ntiles)) {
      __threadfence();
      TileDone* dn = &a.done[id];
      stVol(&dn->tStart, ldVol(&st->tStart));
      stVol(&dn->tEnd, globaltimer());
      __threadfence_system();
      stVol(&dn->seq, ldVol(&st->seq));
      __threadfence_system();
      atomicAdd(&a.q->completed, 1ull);
    }
  }
  VDEV bool finished() { return *(volatile int*)&a.q->stop != 0; }
  VDEV void fail() {
    atomicCAS((int*)&a.ctl->error, 0, (int)vTimeout);
    atomicExch(&a.q->stop, 1);
    __threadfence_system();
  }
};

// a group's ops, tiles assigned statically: CTA j takes j, j + grid, ...
struct BatchSource {
  const TileBatchArgs& b;
  unsigned long long next;
  VDEV long long claim(unsigned long long* tile) {
    if (next >= b.totalTiles) return -1;
    int lo = 0, hi = b.nops - 1;   // the op whose tiles hold `next`
    while (lo < hi) {
      const int mid = (lo + hi + 1) / 2;
      if (b.ops[mid].tileStart <= next) lo = mid;
      else hi = mid - 1;
    }
    *tile = next - b.ops[lo].tileStart;
    next += gridDim.x;
    return lo;
  }
  VDEV void loadReq(long long id, ServeReq* dst) {
    const TileOpDesc& o = b.ops[id];
    dst->coll = o.coll;
    dst->proto = kDirect;
    dst->dtype = o.dtype;
    dst->redop = o.redop;
    dst->nranks = o.nranks;
    dst->nsub = o.nsub;
    dst->root = o.root;
    dst->vec = o.vec;
    dst->count = o.count;
    dst->chunk = o.chunk;
    dst->slotUnits = 0;
    dst->slotBytes = 0;
    dst->inplaceMask = o.inplaceMask;
    for (int r = 0; r < o.nranks; r++) {
      dst->send[r] = b.ptrs[o.ptrBase + r];
      dst->recv[r] = const_cast<void*>(b.ptrs[o.ptrBase + o.nranks + r]);
    }
  }
  VDEV void geom(long long id, unsigned long long tile, TileWork* w) {
    const TileOpDesc& o = b.ops[id];
    if (o.staged) stagedGeom(tile, o.perBlock, o.tileBytes, o.blockBytes, o.ntiles, w);
    else registerGeom(tile, o.tileUnits, o.units, o.ntiles, w);
  }
  VDEV void done(long long) {}
  VDEV bool finished() { return next >= b.totalTiles; }
  VDEV void fail() {
    if (atomicCAS(b.errClaim, 0, (int)vTimeout) == 0) {
      volatile ErrWord* e = b.err;
      e->rank = -1;
      e->channel = (int)blockIdx.x;
      e->where = 4;
      __threadfence_system();
      e->code = (int)vTimeout;
      __threadfence_system();
    }
  }
};

// What a stage slot holds.  Every slot the engine waits on carries one of
// these, and its mbarrier completes for each: data by the bulk loads' bytes,
// the others by a plain arrive of thread 0.
enum { kStageData = 0, kStageReg = 1, kStageIdle = 2, kStageStop = 3 };

struct StageInfo {
  int kind;
  int id, b;
  int endOfTile;            // data: the tile's last sub-tile
  int tail;                 // data: the op's last tile, with an element tail
  unsigned len;             // data: bytes (a multiple of 16)
  unsigned sub;             // data: bytes per input in the stage
  unsigned long long off;   // data: byte offset in the block
  int nseg;                 // data: ring segment runs of the sub-tile
  int seg[kMaxSegRuns];
  unsigned segEnd[kMaxSegRuns];
  TileWork reg;             // register tile
};

constexpr int kMaxPendingDone = kDoneLag + 4;

VDEV void mbarArrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smemU32(bar)) : "memory");
}

// ---- the tile engine: take tiles from `src` until it has none and never
// will; every thread of the CTA calls it.
//
// The stage slots form a ring of kTileStages; sequence index j uses slot
// j mod kTileStages and its mbarrier's phase j / kTileStages.  Thread 0 (the
// producer) fills index j + kTileStages as soon as index j has been folded:
// with the next sub-tile of its current tile (bulk loads), claiming a new
// tile when the current one is done; with a register tile (an unaligned op);
// or, with nothing to claim, with an idle mark (persistent kernel) or the
// stop mark.  Every thread (thread 0 too) folds the indices in order: a data
// stage costs three barriers, and thread 0 refills after the third while the
// others already wait for the next index.
template <class Src>
__device__ void tileEngine(Src& src, unsigned stageBytes, unsigned long long copyTimeoutNs, bool persistent) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ ServeReq sReq[kTileStages];   // the op of each stage
  __shared__ ServeReq sCur;                // the op being issued (thread 0)
  __shared__ StageInfo sInfo[kTileStages];
  unsigned char* in = smem;
  unsigned char* out = smem + (size_t)kTileStages * stageBytes;
  uint64_t* bar = (uint64_t*)(out + 2 * (size_t)kTileOutBytes);

  // thread 0's producer state
  unsigned long long filled = 0;               // sequence indices filled so far
  long long curId = -1;
  unsigned long long curOff = 0, curEnd = 0;
  unsigned curSub = 0;
  int curB = 0, curTail = 0;
  unsigned curGen = 0, stageGen[kTileStages];   // which claim each stage's op copy is of
  for (int i = 0; i < kTileStages; i++) stageGen[i] = ~0u;
  long long doneId[kMaxPendingDone];
  unsigned long long doneGroup[kMaxPendingDone];
  int ndone = 0;
  unsigned idleNs = 64;
  bool stopped = false;

  // thread 0: every pending tile completion, once all store groups are done
  auto flushDone = [&]() {
    bulkWaitAll();
    for (int i = 0; i < ndone; i++) src.done(doneId[i]);
    ndone = 0;
  };
  // thread 0: fill sequence index `filled` (its slot has been folded)
  auto fill = [&]() {
    const int stg = (int)(filled % kTileStages);
    StageInfo& si = sInfo[stg];
    if (stopped) return;   // the stop mark is the last index filled
    if (curId < 0) {
      unsigned long long tl = 0;
      const long long id = src.claim(&tl);
      if (id < 0) {
        flushDone();
        if (src.finished()) {
          si.kind = kStageStop;
          stopped = true;
        } else {
          si.kind = kStageIdle;
          if (persistent) {
            __nanosleep(idleNs);
            idleNs = idleNs < 4096 ? 2 * idleNs : 4096;
          }
        }
        mbarArrive(&bar[stg]);
        filled++;
        return;
      }
      idleNs = 64;
      TileWork w;
      src.geom(id, tl, &w);
      if (!w.staged) {
        si.kind = kStageReg;
        si.id = (int)id;
        si.reg = w;
        src.loadReq(id, &sReq[stg]);   // the slot's own op copy
        stageGen[stg] = ~0u;
        mbarArrive(&bar[stg]);
        filled++;
        return;
      }
      src.loadReq(id, &sCur);
      curId = id;
      curGen++;
      curB = w.b;
      curOff = w.off;
      curEnd = w.end;
      curTail = w.tail && hasTail(&sCur);
      const unsigned nIn = sCur.coll == kAllGather ? 1u : (unsigned)sCur.nranks;
      unsigned sub = stageBytes / nIn;
      sub = sub < kTileOutBytes ? sub : kTileOutBytes;
      curSub = sub & ~127u;
    }
    const unsigned len = (unsigned)(curEnd - curOff < curSub ? curEnd - curOff : curSub);
    si.kind = kStageData;
    si.off = curOff;
    si.len = len;
    si.sub = curSub;
    si.id = (int)curId;
    si.b = curB;
    si.endOfTile = (curOff + len >= curEnd) ? 1 : 0;
    si.tail = si.endOfTile && curTail;
    si.nseg = cutSegments(&sCur, curB, curOff, len, si.seg, si.segEnd);
    if (stageGen[stg] != curGen) {   // the stage holds another claim's op
      sReq[stg] = sCur;
      stageGen[stg] = curGen;
    }
    const ServeReq& r = sCur;
    unsigned char* dst = in + (size_t)stg * stageBytes;
    if (r.coll == kAllGather) {
      mbarExpect(&bar[stg], len);
      bulkLoad(dst, (const char*)r.send[curB] + curOff, len, &bar[stg]);
    } else {
      const unsigned long long esz = (r.dtype == kF16 || r.dtype == kBF16) ? 2 : 4;
      const unsigned long long from =
          (r.coll == kReduceScatter ? (unsigned long long)curB * r.count * esz : 0ull) + curOff;
      mbarExpect(&bar[stg], len * (unsigned)r.nranks);
      for (int q = 0; q < r.nranks; q++)
        bulkLoad(dst + (size_t)q * curSub, (const char*)r.send[q] + from, len, &bar[stg]);
    }
    filled++;
    curOff += len;
    if (curOff >= curEnd) curId = -1;
  };

  if (threadIdx.x == 0) {
    for (int s = 0; s < kTileStages; s++) mbarInit(&bar[s], 1);
    fenceBarrierInit();
    for (int s = 0; s < kTileStages; s++) fill();
  }
  __syncthreads();

  // dsn: data stages folded so far (every thread counts them alike): the
  // output buffer and the store group of a data stage go by it
  unsigned long long dsn = 0;
  for (unsigned long long j = 0;; j++) {
    const int stg = (int)(j % kTileStages);
    const bool ok = stageWait(&bar[stg], (unsigned)((j / kTileStages) & 1ull), copyTimeoutNs);
    if (__syncthreads_or(!ok)) {
      if (threadIdx.x == 0) {
        // loads still in flight must land before the CTA's shared memory is released
        for (unsigned long long q = j; q < filled; q++)
          (void)stageWait(&bar[q % kTileStages], (unsigned)((q / kTileStages) & 1ull), copyTimeoutNs);
        bulkWaitAll();
        src.fail();
      }
      return;
    }
    const int kind = sInfo[stg].kind;
    if (kind == kStageStop) {
      // the data stages before the mark have committed their stores since
      // it was filled: wait for them and report their tiles
      if (threadIdx.x == 0) flushDone();
      return;
    }
    if (kind == kStageIdle) {
      __syncthreads();                // everyone has read the mark
      if (threadIdx.x == 0) fill();
      continue;
    }
    if (kind == kStageReg) {
      // a tile of an unaligned op: the register kernels' paths
      const TileWork w = sInfo[stg].reg;
      const int id = sInfo[stg].id;
      runTile(&sReq[stg], w.lo, w.hi, w.tail != 0);
      __threadfence();
      __syncthreads();
      if (threadIdx.x == 0) {
        src.done(id);
        fill();
      }
      continue;
    }
    // a data stage
    const int ob = (int)(dsn & 1ull);
    if (threadIdx.x == 0) {
      // out[ob] was last read by the store group of data stage dsn - 2,
      // which has read it once at most one group is pending; the tiles
      // whose last group is older than the newest kDoneLag are done
      bulkWaitRead1();
      bulkWaitDoneLag();
      int keep = 0;
      for (int i = 0; i < ndone; i++) {
        if (doneGroup[i] + kDoneLag + 1 <= dsn) {
          src.done(doneId[i]);
        } else {
          doneId[keep] = doneId[i];
          doneGroup[keep] = doneGroup[i];
          keep++;
        }
      }
      ndone = keep;
    }
    __syncthreads();
    const StageInfo si = sInfo[stg];
    const ServeReq* r = &sReq[stg];
    unsigned char* o = out + (size_t)ob * kTileOutBytes;
    foldStageAny(r, (unsigned)((size_t)stg * stageBytes), si.sub, (unsigned)(o - smem), si.len, si.off,
                 si.seg, si.segEnd, si.nseg);
    fenceProxyAsync();
    __syncthreads();   // o written; the stage read by every thread
    if (si.tail) {     // the element tail, with ordinary loads and stores
      tailAny(r);
      __threadfence();
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      if (r->coll == kReduceScatter) {
        bulkStore((char*)r->recv[si.b] + si.off, o, si.len);
      } else {
        const bool ag = r->coll == kAllGather;
        const unsigned long long dst = (ag ? (unsigned long long)si.b * r->count : 0ull) + si.off;
        for (int q = 0; q < r->nranks; q++) {
          if (ag && q == si.b && ((r->inplaceMask >> q) & 1ull)) continue;   // its own block, in place
          bulkStore((char*)r->recv[q] + dst, o, si.len);
        }
      }
      bulkCommit();
      if (si.endOfTile) {
        doneId[ndone] = si.id;
        doneGroup[ndone] = dsn;
        ndone++;
      }
      fill();   // refill this slot: index j + kTileStages
    }
    dsn++;
  }
}

__global__ void __launch_bounds__(kTileThreads, 1) kServeTiles(const __grid_constant__ TileArgs a) {
  if (blockIdx.x == 0) {
    if (threadIdx.x < 32) ingest(a);
    return;
  }
  ServeSource src{a};
  tileEngine(src, a.stageBytes, a.copyTimeoutNs, true);
}

// a group's direct calls in one launch (one CTA per SM)
__global__ void __launch_bounds__(kTileThreads, 1) kBatchTiles(const __grid_constant__ TileBatchArgs b) {
  BatchSource src{b, (unsigned long long)blockIdx.x};
  tileEngine(src, b.stageBytes, b.copyTimeoutNs, false);
}

}  // namespace

const void* serveTilesKernel() { return (const void*)kServeTiles; }
const void* batchTilesKernel() { return (const void*)kBatchTiles; }
int serveTilesThreads() { return kTileThreads; }
int serveTilesUnitsPerIter() { return kTileThreads * kTileNU; }
int serveTilesStages() { return kTileStages; }
unsigned serveTilesOutBytes() { return kTileOutBytes; }
size_t serveTilesSmem(unsigned stageBytes) {
  return (size_t)kTileStages * stageBytes + 2 * (size_t)kTileOutBytes + 8 * (size_t)kTileStages;
}

}  // namespace vc
