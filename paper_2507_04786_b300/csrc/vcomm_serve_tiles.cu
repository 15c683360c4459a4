// vcomm_serve_tiles.cu -- the tile engine: direct-protocol collectives cut
// into tiles and run by resident CTAs, one per SM.  Two kernels use it:
// kBatchTiles runs a group call's direct calls in one launch (the tiles laid
// end to end, CTA j taking tiles j, j + grid, ...), and kServeTiles is
// serving mode 3.
//
// Serving: the host appends requests to a ring in host-mapped memory.  CTA
// 0 of the kernel (one warp) ingests them in order: it copies each entry
// into device state and publishes it on one of two device queues, small
// requests and large ones.  Every other CTA takes the next tile of the first
// request of the small queue that still has tiles, else of the large queue
// (the large queue first when its head was queued well before the small
// queue's head), and folds its 16-byte units exactly as the direct
// protocol's kernels do (each unit's ring chain in the ring schedule's order,
// so the bits are those of a per-call launch with the same plan).  The CTA
// that finishes a request's last tile writes its completion into host-mapped
// memory.  A small request that arrives while a large one runs takes the
// next free CTAs, so it waits for a tile at most; large requests share the
// GPU tile by tile in arrival order.
//
// Data movement.  A tile of a 16-byte aligned request is a byte range of one
// block (AllReduce, Reduce, Broadcast: the buffer; ReduceScatter / AllGather:
// block b) that moves through shared memory in sub-tiles.  A producer warp
// issues bulk asynchronous copies of a sub-tile's inputs (k for a reduction,
// one for a copy; a lane per rank) into one of three stages; eight consumer
// warps fold the stage into an output buffer; the producer bulk-stores it to
// every output.  Producer and consumers meet only on mbarriers, so the
// producer's claims, stores and completions overlap the folds, and the
// stages run ahead across tile boundaries.  ReduceScatter blocks that are
// not whole 16-byte units load a window one unit longer and cut each 16-byte
// piece out of two aligned ones; AllGather blocks that are not whole units
// are stored to their aligned destination units, their edge bytes with
// ordinary stores.  Requests that are not 16-byte aligned take the register
// kernels' element-wise path, one tile at a time.
//
// No CTA waits on another: claims and completions are atomics.  Within a
// CTA every wait is bounded: the producer's idle polls by the ingest's idle
// timeout and the stop word; a consumer's wait for a slot by the producer's
// idle heartbeat and then copyTimeoutNs; the waits for the CTA's own bulk
// copies by copyTimeoutNs; a wait that runs out aborts the whole CTA.
#include <cuda_runtime.h>

#include <cstddef>

#include "vcomm_direct.cuh"
#include "vcomm_kernels.h"

namespace vc {
namespace {

using namespace direct;

constexpr int kTileConsumers = 256;                   // folding threads: warps 0..7
constexpr int kConsumerWarps = kTileConsumers / 32;
constexpr int kTileThreads = kTileConsumers + 32;     // and one producer warp
constexpr int kTileStages = 3;
using Consumers = FirstThreads<kTileConsumers>;
constexpr unsigned kTileOutBytes = 16384;   // one folded sub-tile
constexpr int kTileOutBufs = 2;             // output buffers, used in turn
constexpr int kTileStateWords = (int)(offsetof(TileState, next) / 8);   // request .. klass


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

// ---- register path: ops the staged path does not take (buffers that are
// not 16-byte aligned, blocks of less than a unit or two, AllGather blocks
// that are not whole units).  Reductions go element by element (the host
// gives them vec 0), copies by aligned, shifted or single bytes; one body per
// (dtype, op), out of line, so the engine's own frame stays small.
template <class T, class Op>
__device__ __noinline__ void tileReduce(const ServeReq* q, unsigned long long lo, unsigned long long hi,
                                        bool tail) {
  directReduce<T, Op, Unit1L2<T>, 1, Consumers>(viewOfReq(q), lo, hi, tail);
}

__device__ __noinline__ void tileCopy(const ServeReq* q, unsigned long long lo, unsigned long long hi, bool tail) {
  const DirectView v = viewOfReq(q);
  if (q->vec == 1) directCopy<Unit16L2<uint8_t>, Consumers>(v, lo, hi, tail);
  else if (q->vec == 2) directCopyShifted<L2Mem, Consumers>(v, lo, hi, tail);
  else directCopy<Unit1L2<uint8_t>, Consumers>(v, lo, hi, tail);
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

// ---- staged path: fold one sub-tile from the stage at shared-memory byte
// offset `in` (input q at in + q x stride) into the output buffer at offset
// `o` (offsets into the kernel's dynamic shared memory, read through the
// array itself so the loads are ordinary shared loads), `ulen` bytes.  Unit
// u's chain starts at rank seg[i] + 1 for the first i with u < segEnd[i]
// (thread 0 has cut the sub-tile into its ring segments; nseg == 0: look each
// unit's segment up).  d != 0: every input piece starts d bytes into an
// aligned unit of its window (ReduceScatter blocks that are not whole units)
// and is cut out of two aligned units.
constexpr int kMaxSegRuns = 4;

// a unit's ring segment looked up in the partition (out of line: the fold
// needs it only for sub-tiles that hold many segments)
__device__ __noinline__ int unitSegment(const ServeReq* q, unsigned long long e0, int esz,
                                        unsigned long long* runEnd) {
  return arSegment(viewOfReq(q), e0, esz, runEnd);
}

template <class T, class Op, bool kShift>
__device__ __noinline__ void foldStage(const ServeReq* q, unsigned in, unsigned stride, unsigned o, unsigned ulen,
                                       unsigned long long off, const int* seg, const unsigned* segEnd, int nseg,
                                       unsigned d) {
  extern __shared__ __align__(128) unsigned char smem[];
  const int k = q->nranks;
  unsigned long long runEnd = 0;   // nseg == 0: each unit's segment from the partition
  int s0 = 0;
  for (unsigned u = threadIdx.x * 16u; u < ulen; u += kTileConsumers * 16u) {
    int s;
    if (nseg > 0) {
      int i = 0;
      while (i + 1 < nseg && u >= segEnd[i]) i++;
      s = seg[i];
    } else {
      const unsigned long long e0 = (off + u) / sizeof(T);
      if (e0 >= runEnd) s0 = unitSegment(q, e0, (int)sizeof(T), &runEnd);
      s = s0;
    }
    int r = s + 1 < k ? s + 1 : 0;
    const unsigned char* base = smem + in + u;
    auto piece = [&](int rr) {
      const unsigned char* p = base + (unsigned)rr * stride;
      if (kShift) return shiftBytes(*(const uint4*)p, *(const uint4*)(p + 16), d);
      return *(const uint4*)p;
    };
    uint4 acc = piece(r);
#pragma unroll 4
    for (int j = 1; j < k; j++) {
      if (++r == k) r = 0;
      acc = combine<T, Op, uint4>(acc, piece(r));
    }
    *(uint4*)(smem + o + u) = acc;
  }
}

// a copy's stage into the output buffer; d != 0: each 16-byte piece starts
// d bytes into the window (AllGather blocks that are not whole units, whose
// destination units are aligned)
__device__ __forceinline__ void copyStage(unsigned in, unsigned o, unsigned len, unsigned d) {
  extern __shared__ __align__(128) unsigned char smem[];
  for (unsigned u = threadIdx.x * 16u; u < len; u += kTileConsumers * 16u) {
    const unsigned char* p = smem + in + u;
    *(uint4*)(smem + o + u) = d ? shiftBytes(*(const uint4*)p, *(const uint4*)(p + 16), d) : *(const uint4*)p;
  }
}

VDEV bool copyColl(int coll) { return coll == kAllGather || coll == kBroadcast; }

VDEV void foldStageAny(const ServeReq* q, unsigned in, unsigned stride, unsigned o, unsigned ulen,
                       unsigned long long off, const int* seg, const unsigned* segEnd, int nseg, unsigned d) {
  if (copyColl(q->coll)) {   // a copy: the one input as it is
    copyStage(in, o, ulen, d);
    return;
  }
  const bool mx = q->redop == kMax;
#define VC_FOLD(T)                                                                                  \
  d ? (mx ? foldStage<T, OpMax, true>(q, in, stride, o, ulen, off, seg, segEnd, nseg, d)               \
          : foldStage<T, OpSum, true>(q, in, stride, o, ulen, off, seg, segEnd, nseg, d))              \
    : (mx ? foldStage<T, OpMax, false>(q, in, stride, o, ulen, off, seg, segEnd, nseg, d)              \
          : foldStage<T, OpSum, false>(q, in, stride, o, ulen, off, seg, segEnd, nseg, d))
  if (q->dtype == kI32) VC_FOLD(int32_t);
  else if (q->dtype == kF32) VC_FOLD(float);
  else if (q->dtype == kF16) VC_FOLD(__half);
  else VC_FOLD(__nv_bfloat16);
#undef VC_FOLD
}

// producer: the ring segments of a sub-tile (bytes [off, off + len) of block
// b): AllReduce segments from the partition (a segment is normally a chunk,
// far longer than a sub-tile; 0 runs if the sub-tile holds more than
// kMaxSegRuns, as the short segments of a small buffer's last loop do, and
// the fold then looks each unit's segment up); a ReduceScatter block b is one
// run starting at rank b + 1, a Reduce one starting at root + 1.  The run
// found last is kept in `cache` ([lo, hi) bytes, segment s, for claim gen):
// a tile's sub-tiles come in rising order, so most of them lie inside it
// and need no partition arithmetic.
struct SegCache {
  unsigned long long lo, hi;
  int s;
  unsigned gen;
};
VDEV int cutSegments(const ServeReq* q, int b, unsigned long long off, unsigned len, int* seg, unsigned* segEnd,
                     SegCache& cache, unsigned gen) {
  if (q->coll != kAllReduce) {
    seg[0] = q->coll == kReduce ? q->root : b;
    segEnd[0] = len;
    return 1;
  }
  const unsigned long long esz = (q->dtype == kF16 || q->dtype == kBF16) ? 2 : 4;
  unsigned u = 0;
  int n = 0;
  while (u < len) {
    if (n == kMaxSegRuns) return 0;
    const unsigned long long x = off + u;
    if (cache.gen != gen || x < cache.lo || x >= cache.hi) {
      unsigned long long runEnd;   // in elements
      cache.s = arSegment(viewOfReq(q), x / esz, (int)esz, &runEnd);
      cache.lo = x;
      cache.hi = runEnd * esz;
      cache.gen = gen;
    }
    seg[n] = cache.s;
    const unsigned long long endB = cache.hi - off;
    segEnd[n] = endB < len ? (unsigned)endB : len;
    u = segEnd[n];
    n++;
  }
  return n;
}

// ---- the elements a staged op leaves to ordinary loads and stores, done
// with its last tile: the element tail after the last full unit (AllReduce,
// Reduce: of the buffer; ReduceScatter: of every block) and, for a
// ReduceScatter of blocks that are not whole units, the last block's last
// full unit (its window would reach past the end of the send buffers)
template <class T, class Op>
__device__ __noinline__ void tailReduce(const ServeReq* q) {
  const DirectView v = viewOfReq(q);
  const int k = q->nranks;
  constexpr unsigned long long E = 16 / sizeof(T);
  const unsigned long long nunit = q->count / E;
  if (q->coll == kReduceScatter) {
    for (int b = 0; b < k; b++) {
      const unsigned long long from = (b == k - 1 && q->vec == 2 && nunit > 0) ? (nunit - 1) * E : nunit * E;
      for (unsigned long long i = from + threadIdx.x; i < q->count; i += kTileConsumers) {
        const T x = foldChain<T, Op, Unit1L2<T>>(v, b, ((unsigned long long)b * q->count + i) * sizeof(T));
        *(T*)((char*)v.recv[b] + i * sizeof(T)) = x;
      }
    }
    return;
  }
  for (unsigned long long i = nunit * E + threadIdx.x; i < q->count; i += kTileConsumers) {
    unsigned long long re;
    const int s = q->coll == kReduce ? q->root : arSegment(v, i, (int)sizeof(T), &re);
    const T x = foldChain<T, Op, Unit1L2<T>>(v, s, i * sizeof(T));
    if (q->coll == kReduce) *(T*)((char*)v.recv[q->root] + i * sizeof(T)) = x;
    else
      for (int r = 0; r < k; r++) *(T*)((char*)v.recv[r] + i * sizeof(T)) = x;
  }
}

// the bytes of an AllGather block (count bytes, not whole units) that the
// staged path leaves out: before its first aligned destination unit and
// after the agStaged bytes that follow it
VDEV unsigned long long agLead(unsigned long long b, unsigned long long count) {
  return (16 - ((b * count) & 15)) & 15;
}
VDEV unsigned long long agStaged(unsigned long long count) { return count / 16 * 16 - 16; }

VDEV void tailAny(const ServeReq* q) {
  if (q->coll == kAllGather) {   // shifted blocks: each block's edge bytes
    const unsigned long long B = q->count, W = agStaged(B);
    const int k = q->nranks;
    for (int b = 0; b < k; b++) {
      const unsigned long long lead = agLead((unsigned long long)b, B);
      const unsigned long long nedge = B - W;   // lead bytes, then the rest after lead + W
      for (unsigned long long t = threadIdx.x; t < nedge; t += kTileConsumers) {
        const unsigned long long x = t < lead ? t : W + t;   // source offset in block b
        const uint8_t c = Unit1L2<uint8_t>::load((const char*)q->send[b] + x);
        for (int r = 0; r < k; r++) ((uint8_t*)q->recv[r])[(unsigned long long)b * B + x] = c;
      }
    }
    return;
  }
  if (q->coll == kBroadcast) {   // the bytes after the last full unit
    const unsigned long long from = q->count / 16 * 16;
    for (unsigned long long i = from + threadIdx.x; i < q->count; i += kTileConsumers) {
      const uint8_t c = Unit1L2<uint8_t>::load((const char*)q->send[q->root] + i);
      for (int r = 0; r < q->nranks; r++)
        if (!(r == q->root && ((q->inplaceMask >> r) & 1ull))) ((uint8_t*)q->recv[r])[i] = c;
    }
    return;
  }
  const bool mx = q->redop == kMax;
  if (q->dtype == kI32) mx ? tailReduce<int32_t, OpMax>(q) : tailReduce<int32_t, OpSum>(q);
  else if (q->dtype == kF32) mx ? tailReduce<float, OpMax>(q) : tailReduce<float, OpSum>(q);
  else if (q->dtype == kF16) mx ? tailReduce<__half, OpMax>(q) : tailReduce<__half, OpSum>(q);
  else mx ? tailReduce<__nv_bfloat16, OpMax>(q) : tailReduce<__nv_bfloat16, OpSum>(q);
}

VDEV bool hasTail(const ServeReq* q) {
  if (q->coll == kAllGather) return q->vec == 2;       // staged blocks of whole units have none
  if (q->coll == kBroadcast) return q->count % 16 != 0;
  if (q->coll == kReduceScatter && q->vec == 2) return true;
  const unsigned long long E = (q->dtype == kF16 || q->dtype == kBF16) ? 8 : 4;
  return q->count % E != 0;
}

// Small requests go first, as long as they do not starve a large one: when
// the large queue's head was ingested this much earlier than the small
// queue's head, the large queue goes first.
constexpr unsigned long long kLargeUrgentNs = 500000;
constexpr unsigned long long kAgeCheckNs = 20000;   // how often the ingester compares the heads

// ---- CTA 0, warp 0: ingest ring entries firstSeq, firstSeq + 1, ... in order
__device__ void ingest(const TileArgs& a) {
  const int lane = threadIdx.x & 31;
  TileQueues* q = a.q;
  volatile TileCtl* ctl = a.ctl;
  unsigned long long next = a.firstSeq;
  uint64_t idle0 = globaltimer(), drain0 = 0, lastAge = 0;
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
      const uint64_t now = lane == 0 ? globaltimer() : 0;
      if (lane == 0 && now - lastAge > kAgeCheckNs) {   // between arrivals: compare the two queues' heads
        lastAge = now;
        unsigned long long ts[2] = {0, 0};   // ingest times of the heads (0: none)
        for (int c = 0; c < 2; c++) {
          const unsigned long long h = ldVol(&q->head[c]), t = ldVol(&q->tail[c]);
          if (h < t) {
            const unsigned long long en = ldVol(&q->entry[c][h % kTileRing]);
            if ((en >> 32) == (h & 0xffffffffull)) ts[c] = ldVol(&a.state[(int)(en & 0xffffffffull) - 1].tStart);
          }
        }
        const unsigned long long urgent = (ts[0] && ts[1] && ts[1] + kLargeUrgentNs < ts[0]) ? 1 : 0;
        if (urgent != ldVol(&q->urgent)) stVol(&q->urgent, urgent);
      }
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

// ---- where tiles come from.  The engine below calls a source from its
// producer warp:
//   take(&w, dst, scratch, lane)
//                       (every lane) claim the next tile: its op id (>= 0, or
//                       -1: none now), the op's description into shared
//                       memory (dst) and the tile's work (w): a byte range of
//                       one block (staged), or a range of the register
//                       kernels' units
//   (lane 0)
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
  static constexpr bool kReportsDone = true;
  const TileArgs& a;
  // lane 0 finds the first queued request that may have tiles left and
  // claims a tile of it with an atomic; meanwhile every lane fetches that
  // request's state (request and geometry) into `scratch`, a word per lane
  // at a time, so the claim and the fetch take one round trip together.  A
  // claim past the request's last tile moves the queue's head on and tries
  // the next request.
  VDEV long long take(TileWork* w, ServeReq* dst, unsigned long long* scratch, int lane) {
    TileQueues* q = a.q;
    int c = 0, tries = 0;
    if (lane == 0) c = ldVol(&q->urgent) ? 1 : 0;   // the large queue first when its head starves
    c = __shfl_sync(0xffffffffu, c, 0);
    while (tries < 2) {
      int s = -1;
      unsigned long long h = 0, tl = 0;
      if (lane == 0) {
        h = ldVol(&q->head[c]);
        const unsigned long long t = ldAcquire(&q->tail[c]);
        if (h < t) {
          const unsigned long long en = ldVol(&q->entry[c][h % kTileRing]);
          if ((en >> 32) == (h & 0xffffffffull)) {   // (always, once the tail is past it)
            s = (int)(en & 0xffffffffull) - 1;
            tl = atomicAdd(&a.state[s].next, 1ull);
          }
        }
      }
      s = __shfl_sync(0xffffffffu, s, 0);
      if (s < 0) {   // this queue is empty: the other one
        c ^= 1;
        tries++;
        continue;
      }
      const unsigned long long* src = (const unsigned long long*)&a.state[s];
      for (int i = lane; i < kTileStateWords; i += 32) scratch[i] = ldVol(&src[i]);
      tl = __shfl_sync(0xffffffffu, tl, 0);
      __syncwarp();
      const TileState* st = (const TileState*)scratch;
      if (tl < st->ntiles) {
        for (int i = lane; i < (int)(sizeof(ServeReq) / 8); i += 32)
          ((unsigned long long*)dst)[i] = ((const unsigned long long*)&st->req)[i];
        if (lane == 0) {
          if (st->staged) stagedGeom(tl, st->perBlock, st->tileBytes, st->blockBytes, st->ntiles, w);
          else registerGeom(tl, st->tileUnits, st->units, st->ntiles, w);
        }
        __syncwarp();
        return s;
      }
      if (lane == 0) atomicCAS(&q->head[c], h, h + 1);   // every tile of entry h is claimed
      __syncwarp();
    }
    return -1;
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
  static constexpr bool kReportsDone = false;   // the launch's end is the group's completion
  const TileBatchArgs& b;
  unsigned long long next;
  // lane 0: the op whose tiles hold `next`, its description from the
  // launch's parameters and the tile's work
  VDEV long long take(TileWork* w, ServeReq* dst, unsigned long long*, int lane) {
    long long id = -1;
    if (lane == 0 && next < b.totalTiles) {
      int lo = 0, hi = b.nops - 1;
      while (lo < hi) {
        const int mid = (lo + hi + 1) / 2;
        if (b.ops[mid].tileStart <= next) lo = mid;
        else hi = mid - 1;
      }
      id = lo;
      const unsigned long long tile = next - b.ops[lo].tileStart;
      next += gridDim.x;
      const TileOpDesc& o = b.ops[lo];
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
      if (o.staged) stagedGeom(tile, o.perBlock, o.tileBytes, o.blockBytes, o.ntiles, w);
      else registerGeom(tile, o.tileUnits, o.units, o.ntiles, w);
    }
    id = (long long)__shfl_sync(0xffffffffu, (unsigned long long)id, 0);
    __syncwarp();
    return id;
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

// What a stage slot holds.  Every slot the consumers wait on carries one of
// these, and its `full` mbarrier completes for each: data by the bulk loads'
// bytes, the others by a plain arrive of the producer.
enum { kStageData = 0, kStageReg = 1, kStageStop = 2 };

struct StageInfo {
  int kind;
  int id, b;
  int endOfTile;            // data: the tile's last sub-tile
  int tail;                 // data: the op's last tile, with an element tail
  unsigned len;             // data: bytes (a multiple of 16)
  unsigned ulen;            // data: bytes folded and stored (len, or len - 16: the last
                            // unit of a shifted op's last sub-tile goes with the tail)
  unsigned stride;          // data: bytes per input in the stage
  unsigned d;               // data: shifted inputs start d bytes into their window
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

// The producer's state (kept in shared memory: the thread's local memory
// mostly lives in L2 when shared memory takes the SM's on-chip storage).
struct Producer {
  unsigned long long filled;                  // sequence indices filled so far
  unsigned long long groups;                  // store groups committed (data stages retired)
  long long curId;                            // the tile being issued (-1: none)
  unsigned long long curOff, curEnd;
  unsigned curSub, curStride, curD, curGen;
  int curB, curTail;
  unsigned stageGen[kTileStages];             // which claim each stage's op copy is of
  SegCache seg;                               // the ring segment run found last
  long long doneId[kMaxPendingDone];          // finished tiles, completion unconfirmed
  unsigned long long doneGroup[kMaxPendingDone];
  int ndone;
  int stopped;
};

struct EngineSmem {
  ServeReq sReq[kTileStages];   // the op of each stage
  ServeReq sCur;                // the op being issued
  TileWork work;                // the claimed tile's work
  unsigned long long scratch[kTileStateWords];   // a claimed op's state, as fetched
  StageInfo sInfo[kTileStages];
  Producer p;
  uint64_t full[kTileStages];   // a slot is filled (producer / bulk loads)
  uint64_t empty[kTileStages];  // a slot is consumed (one arrive per consumer warp)
  uint64_t outFree[kTileOutBufs];   // an output buffer's store group has read it
  int abort;                    // a wait ran out: everyone leaves
  unsigned beat;                // the producer's idle polls (it is alive, with nothing to claim)
};

VDEV bool aborted(const EngineSmem& e) { return *(const volatile int*)&e.abort != 0; }
VDEV void setAbort(EngineSmem& e) { *(volatile int*)&e.abort = 1; }

// wait for phase `parity` of *bar; false once the engine aborts or after timeoutNs
VDEV bool engineWait(uint64_t* bar, unsigned parity, unsigned long long timeoutNs, const EngineSmem& e) {
  if (mbarTryWait(bar, parity)) return true;
  const uint64_t t0 = globaltimer();
  while (true) {
    if (mbarTryWait(bar, parity)) return true;
    if (aborted(e) || globaltimer() - t0 > timeoutNs) return false;
  }
}

// The producer is one warp.  Lane 0 makes every decision (claims, the
// slots' contents, completions) in shared memory; the bulk copies of a slot
// are spread over the lanes, lane q taking ranks q, q + 32, ... (a bulk
// group belongs to the thread that commits it, so every lane commits one
// group per data stage, and waits for its own).
constexpr unsigned kFullMask = 0xffffffffu;

// consumers: wait for sequence index j.  While the producer has not filled
// it (nothing to claim yet) the wait lasts as long as the producer keeps
// polling; once filled, its bulk loads have timeoutNs to land.
VDEV bool waitFull(EngineSmem& e, unsigned long long j, unsigned long long timeoutNs) {
  uint64_t* bar = &e.full[j % kTileStages];
  const unsigned parity = (unsigned)((j / kTileStages) & 1ull);
  if (mbarTryWait(bar, parity)) return true;
  uint64_t t0 = globaltimer();
  unsigned beat = *(const volatile unsigned*)&e.beat;
  bool filled = false;
  while (true) {
    if (mbarTryWait(bar, parity)) return true;
    if (aborted(e)) return false;
    const uint64_t now = globaltimer();
    if (!filled) {
      const unsigned b = *(const volatile unsigned*)&e.beat;
      if (*(const volatile unsigned long long*)&e.p.filled > j) {
        filled = true;
        t0 = now;
      } else if (b != beat) {
        beat = b;
        t0 = now;
      }
    }
    if (now - t0 > timeoutNs) return false;
  }
}

// producer warp: every store group has completed; lane 0 reports the
// pending tiles
template <class Src>
VDEV void flushDone(Src& src, Producer& p, int lane) {
  bulkWaitAll();
  fenceProxyGlobal();   // this lane's completed bulk writes, before the reports
  __syncwarp();
  if (lane == 0) {
    for (int i = 0; i < p.ndone; i++) src.done(p.doneId[i]);
    p.ndone = 0;
  }
  __syncwarp();
}

// producer warp: fill sequence index p.filled (its slot has been consumed);
// false: nothing to claim right now (no slot filled)
template <class Src>
__device__ __forceinline__ bool fillStage(Src& src, EngineSmem& e, unsigned char* in, unsigned stageBytes, int lane) {
  Producer& p = e.p;
  if (p.stopped) return true;   // the stop mark is the last index filled
  const int stg = (int)(p.filled % kTileStages);
  StageInfo& si = e.sInfo[stg];
  uint64_t* bar = &e.full[stg];
  if (p.curId < 0) {
    // no staged tile is in progress: sCur is free for the next one
    const long long id = src.take(&e.work, &e.sCur, e.scratch, lane);
    if (id < 0) {
      int fin = 0;
      if (lane == 0) fin = src.finished() ? 1 : 0;
      if (!__shfl_sync(kFullMask, fin, 0)) return false;
      flushDone(src, p, lane);
      if (lane == 0) {
        si.kind = kStageStop;
        p.stopped = 1;
        mbarArrive(bar);
        p.filled++;
      }
      __syncwarp();
      return true;
    }
    int staged = 0;
    if (lane == 0) {
      const TileWork w = e.work;
      staged = w.staged;
      if (!w.staged) {
        si.kind = kStageReg;
        si.id = (int)id;
        si.reg = w;
        e.sReq[stg] = e.sCur;   // the slot's own op copy
        p.stageGen[stg] = ~0u;
        mbarArrive(bar);
        p.filled++;
      } else {
        p.curId = id;
        p.curGen++;
        p.curB = w.b;
        p.curOff = w.off;
        p.curEnd = w.end;
        p.curTail = w.tail && hasTail(&e.sCur);
        const ServeReq& r = e.sCur;
        const unsigned nIn = copyColl(r.coll) ? 1u : (unsigned)r.nranks;
        const unsigned pad = r.vec == 2 ? 16u : 0u;   // a shifted window is one unit longer
        unsigned sub = stageBytes / nIn - pad;
        sub = sub < kTileOutBytes ? sub : kTileOutBytes;
        sub &= ~127u;
        // sub-tiles of about equal size, whole 128-byte lines (bulk copies
        // of aligned lines)
        const unsigned long long tb = w.end - w.off;
        const unsigned long long m = (tb + sub - 1) / sub;
        const unsigned long long even = ((tb + m - 1) / m + 127) / 128 * 128;
        p.curSub = (unsigned)(even < sub ? even : sub);
        p.curStride = p.curSub + pad;
        const unsigned long long esz = (r.dtype == kF16 || r.dtype == kBF16) ? 2 : 4;
        if (r.vec != 2) p.curD = 0;
    else if (r.coll == kAllGather) p.curD = (unsigned)agLead((unsigned long long)w.b, r.count);
    else p.curD = (unsigned)(((unsigned long long)w.b * r.count * esz) & 15ull);
      }
    }
    staged = __shfl_sync(kFullMask, staged, 0);
    if (!staged) {
      __syncwarp();
      return true;
    }
  }
  const ServeReq& r = e.sCur;
  unsigned wlen = 0;
  if (lane == 0) {
    const unsigned long long off = p.curOff;
    const unsigned len = (unsigned)(p.curEnd - off < p.curSub ? p.curEnd - off : p.curSub);
    si.kind = kStageData;
    si.off = off;
    si.len = len;
    si.stride = p.curStride;
    si.d = p.curD;
    si.id = (int)p.curId;
    si.b = p.curB;
    si.endOfTile = (off + len >= p.curEnd) ? 1 : 0;
    si.tail = si.endOfTile && p.curTail;
    // a shifted ReduceScatter's very last unit: its window would reach past the end of
    // the send buffers; the tail folds it with element loads
    const bool skipLast = r.vec == 2 && r.coll == kReduceScatter && si.tail;
    si.ulen = skipLast ? len - 16 : len;
    si.nseg = cutSegments(&r, si.b, off, len, si.seg, si.segEnd, p.seg, p.curGen);
    if (p.stageGen[stg] != p.curGen) {   // the stage holds another claim's op
      e.sReq[stg] = r;
      p.stageGen[stg] = p.curGen;
    }
    wlen = (si.d != 0 && !skipLast) ? len + 16 : len;
    mbarExpect(bar, copyColl(r.coll) ? wlen : wlen * (unsigned)r.nranks);
  }
  wlen = __shfl_sync(kFullMask, wlen, 0);
  __syncwarp();   // si and sCur as lane 0 wrote them
  unsigned char* dst = in + (size_t)stg * stageBytes;
  const unsigned long long off = si.off;
  if (copyColl(r.coll)) {   // AllGather: block b of rank b; Broadcast: the root's buffer
    if (lane == 0) bulkLoad(dst, (const char*)r.send[r.coll == kAllGather ? si.b : r.root] + off, wlen, bar);
  } else {
    const unsigned long long esz = (r.dtype == kF16 || r.dtype == kBF16) ? 2 : 4;
    const unsigned long long from =
        (r.coll == kReduceScatter ? (unsigned long long)si.b * r.count * esz : 0ull) + off - si.d;
    for (int q = lane; q < r.nranks; q += 32)
      bulkLoad(dst + (size_t)q * si.stride, (const char*)r.send[q] + from, wlen, bar);
  }
  __syncwarp();   // every lane has read sCur and si
  if (lane == 0) {
    p.filled++;
    p.curOff = off + si.len;
    if (p.curOff >= p.curEnd) p.curId = -1;
  }
  __syncwarp();
  return true;
}

// producer warp: sequence index i has been consumed; a data stage's output
// buffer goes to its outputs as store group n = p.groups (returned; -1 for
// the other kinds of slot)
template <class Src>
__device__ __forceinline__ long long retire(Src& src, EngineSmem& e, unsigned char* out, unsigned long long i,
                                         unsigned long long timeoutNs, int lane, bool* ok) {
  Producer& p = e.p;
  const int stg = (int)(i % kTileStages);
  const bool got = engineWait(&e.empty[stg], (unsigned)((i / kTileStages) & 1ull), timeoutNs, e);
  *ok = __all_sync(kFullMask, got);
  if (!*ok) return -1;
  const StageInfo& si = e.sInfo[stg];
  if (si.kind == kStageReg) {   // the consumers fenced their stores before arriving
    if (lane == 0) src.done(si.id);
    __syncwarp();
    return -1;
  }
  if (si.kind != kStageData) return -1;
  const unsigned long long n = p.groups;
  const ServeReq* r = &e.sReq[stg];
  unsigned char* o = out + (size_t)(n % kTileOutBufs) * kTileOutBytes;
  if (si.ulen > 0) {
    const int c = r->coll;
    if (c == kReduceScatter || c == kReduce) {
      if (lane == 0) bulkStore((char*)r->recv[c == kReduce ? r->root : si.b] + si.off, o, si.ulen);
    } else {
      // AllReduce: every rank; AllGather: block b of every rank; Broadcast:
      // every rank (a rank whose output is its input in place is skipped)
      const int self = c == kAllGather ? si.b : (c == kBroadcast ? r->root : -1);
      // (a shifted AllGather block: from its first aligned destination unit)
      const unsigned long long bb = (unsigned long long)si.b;
      const unsigned long long dst =
          (c == kAllGather ? bb * r->count + (r->vec == 2 ? agLead(bb, r->count) : 0ull) : 0ull) + si.off;
      for (int q = lane; q < r->nranks; q += 32) {
        if (q == self && ((r->inplaceMask >> q) & 1ull)) continue;
        bulkStore((char*)r->recv[q] + dst, o, si.ulen);
      }
    }
  }
  bulkCommit();
  __syncwarp();
  if (lane == 0) {
    p.groups = n + 1;
    if (Src::kReportsDone && si.endOfTile) {
      p.doneId[p.ndone] = si.id;
      p.doneGroup[p.ndone] = n;
      p.ndone++;
    }
  }
  __syncwarp();
  return (long long)n;
}

// producer warp, after store group n was committed: once group
// n + 1 - kTileOutBufs has read its buffer the consumers may write it again;
// the tiles whose last group is older than the newest kDoneLag are reported
template <class Src>
__device__ __forceinline__ void release(Src& src, EngineSmem& e, unsigned long long n, int lane) {
  Producer& p = e.p;
  // every group but the newest kTileOutBufs - 1 has read its buffer
  asm volatile("cp.async.bulk.wait_group.read %0;" ::"n"(kTileOutBufs - 1) : "memory");
  __syncwarp();
  if (lane == 0 && n + 1 >= (unsigned long long)kTileOutBufs)
    mbarArrive(&e.outFree[(n + 1 - kTileOutBufs) % kTileOutBufs]);
  if (Src::kReportsDone) {
    bulkWaitDoneLag();
    fenceProxyGlobal();
    __syncwarp();
    if (lane == 0) {
      int keep = 0;
      for (int j = 0; j < p.ndone; j++) {
        if (p.doneGroup[j] + kDoneLag <= n) {
          src.done(p.doneId[j]);
        } else {
          p.doneId[keep] = p.doneId[j];
          p.doneGroup[keep] = p.doneGroup[j];
          keep++;
        }
      }
      p.ndone = keep;
    }
  }
  __syncwarp();
}

// ---- the producer warp: fill the slots ahead of the consumers, retire each
// slot once consumed, until the stop mark; then retire the rest and report
// the last completions.  A wait that runs out (a bulk load that never lands,
// consumers that left) aborts the engine: the loads still in flight land
// before the warp leaves, and the source records the failure.
template <class Src>
__device__ __noinline__ void produce(Src& src, EngineSmem& e, unsigned char* in, unsigned char* out,
                                     unsigned stageBytes, unsigned long long timeoutNs) {
  const int lane = threadIdx.x & 31;
  Producer& p = e.p;
  if (lane == 0) {
    p.filled = p.groups = 0;
    p.curId = -1;
    p.curOff = p.curEnd = 0;
    p.curSub = p.curStride = p.curD = p.curGen = 0;
    p.curB = p.curTail = 0;
    for (int i = 0; i < kTileStages; i++) p.stageGen[i] = ~0u;
    p.seg.gen = ~0u;
    p.ndone = 0;
    p.stopped = 0;
  }
  __syncwarp();
  unsigned long long retired = 0;
  unsigned idleNs = 32;
  bool ok = true;
  while (!p.stopped) {
    long long n = -1;
    if (p.filled - retired == (unsigned long long)kTileStages) {
      n = retire(src, e, out, retired, timeoutNs, lane, &ok);
      if (!ok) break;
      retired++;
    }
    // the output buffer first: consumers may be waiting for it
    if (n >= 0) release(src, e, (unsigned long long)n, lane);
    if (fillStage(src, e, in, stageBytes, lane)) {
      idleNs = 32;
      continue;
    }
    // nothing to claim: retire what the consumers still hold (their stores
    // and completions go out now), report, and poll again a little later
    while (ok && retired < p.filled) {
      n = retire(src, e, out, retired, timeoutNs, lane, &ok);
      if (!ok) break;
      retired++;
      if (n >= 0) release(src, e, (unsigned long long)n, lane);
    }
    if (!ok) break;
    flushDone(src, p, lane);
    __nanosleep(idleNs);
    idleNs = idleNs < 512 ? 2 * idleNs : 512;
    if (lane == 0) *(volatile unsigned*)&e.beat = *(volatile unsigned*)&e.beat + 1;
  }
  while (ok && retired + 1 < p.filled) {   // every index before the stop mark
    const long long n = retire(src, e, out, retired, timeoutNs, lane, &ok);
    if (!ok) break;
    retired++;
    if (n >= 0) release(src, e, (unsigned long long)n, lane);
  }
  if (ok) {
    flushDone(src, p, lane);
    return;
  }
  if (lane == 0) {
    setAbort(e);
    for (unsigned long long q = retired; q < p.filled; q++)
      if (e.sInfo[q % kTileStages].kind == kStageData)
        (void)stageWait(&e.full[q % kTileStages], (unsigned)((q / kTileStages) & 1ull), timeoutNs);
  }
  bulkWaitAll();
  __syncwarp();
  if (lane == 0) src.fail();
}

// ---- the consumers (warps 0 .. kConsumerWarps - 1): every sequence index in
// order.  A data stage folds into output buffer dsn mod kTileOutBufs (once
// the buffer's previous store group has read it); the op's last sub-tile also does
// the element tail with ordinary loads and stores.  Each warp arrives on the
// slot's `empty` barrier when done with it.
__device__ __noinline__ void consume(EngineSmem& e, unsigned char* out, unsigned stageBytes, unsigned long long timeoutNs) {
  extern __shared__ __align__(128) unsigned char smem[];
  const int lane = threadIdx.x & 31;
  unsigned long long dsn = 0;
  for (unsigned long long j = 0;; j++) {
    const int stg = (int)(j % kTileStages);
    if (!waitFull(e, j, timeoutNs)) {
      setAbort(e);
      return;
    }
    const StageInfo& si = e.sInfo[stg];
    const int kind = si.kind;
    if (kind == kStageStop) return;
    if (kind == kStageReg) {   // a tile the staged path does not take
      runTile(&e.sReq[stg], si.reg.lo, si.reg.hi, si.reg.tail != 0);
      __threadfence();
    } else if (kind == kStageData) {
      const unsigned long long n = dsn++;
      const int ob = (int)(n % kTileOutBufs);
      // the buffer's previous store group (data stage n - kTileOutBufs) has read it
      if (n >= (unsigned long long)kTileOutBufs &&
          !engineWait(&e.outFree[ob], (unsigned)((n / kTileOutBufs - 1) & 1ull), timeoutNs, e)) {
        setAbort(e);
        return;
      }
      const ServeReq* r = &e.sReq[stg];
      unsigned char* o = out + (size_t)ob * kTileOutBytes;
      foldStageAny(r, (unsigned)((size_t)stg * stageBytes), si.stride, (unsigned)(o - smem), si.ulen, si.off,
                   si.seg, si.segEnd, si.nseg, si.d);
      if (si.tail) {   // the element tail, with ordinary loads and stores
        tailAny(r);
        __threadfence();
      }
      fenceProxyAsync();   // this thread's output writes, before the bulk stores read them
    }
    __syncwarp();
    if (lane == 0) mbarArrive(&e.empty[stg]);
  }
}

// ---- the tile engine: take tiles from `src` until it has none and never
// will.  The stage slots form a ring of kTileStages; sequence index j uses
// slot j mod kTileStages and its barriers' phase j / kTileStages.  The
// producer warp runs ahead of the consumer warps by up to kTileStages
// indices, so bulk loads stay in flight while the consumers fold and the
// producer's own work (claims, stores, completions) overlaps theirs.  With
// nothing to claim the producer fills no slot: it retires what the
// consumers hold, reports, and polls again, so a new tile starts at once.
template <class Src>
__device__ void tileEngine(Src& src, unsigned stageBytes, unsigned long long copyTimeoutNs) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ EngineSmem e;
  unsigned char* in = smem;
  unsigned char* out = smem + (size_t)kTileStages * stageBytes;
  if (threadIdx.x == 0) {
    for (int i = 0; i < kTileStages; i++) {
      mbarInit(&e.full[i], 1);
      mbarInit(&e.empty[i], kConsumerWarps);
    }
    for (int i = 0; i < kTileOutBufs; i++) mbarInit(&e.outFree[i], 1);
    e.abort = 0;
    e.beat = 0;
    e.p.filled = 0;
    fenceBarrierInit();
  }
  __syncthreads();
  if (threadIdx.x >= kTileConsumers) {
    produce(src, e, in, out, stageBytes, copyTimeoutNs);
    return;
  }
  consume(e, out, stageBytes, copyTimeoutNs);
}

__global__ void __launch_bounds__(kTileThreads, 1) kServeTiles(const __grid_constant__ TileArgs a) {
  if (blockIdx.x == 0) {
    if (threadIdx.x < 32) ingest(a);
    return;
  }
  ServeSource src{a};
  tileEngine(src, a.stageBytes, a.copyTimeoutNs);
}

// a group's direct calls in one launch (one CTA per SM)
__global__ void __launch_bounds__(kTileThreads, 1) kBatchTiles(const __grid_constant__ TileBatchArgs b) {
  BatchSource src{b, (unsigned long long)blockIdx.x};
  tileEngine(src, b.stageBytes, b.copyTimeoutNs);
}

}  // namespace

const void* serveTilesKernel() { return (const void*)kServeTiles; }
const void* batchTilesKernel() { return (const void*)kBatchTiles; }
int serveTilesThreads() { return kTileThreads; }
int serveTilesUnitsPerIter() { return kTileConsumers; }
int serveTilesStages() { return kTileStages; }
unsigned serveTilesOutBytes() { return kTileOutBytes; }
size_t serveTilesSmem(unsigned stageBytes) {
  return (size_t)kTileStages * stageBytes + (size_t)kTileOutBufs * kTileOutBytes;
}

}  // namespace vc
