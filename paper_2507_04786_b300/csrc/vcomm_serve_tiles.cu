// vcomm_serve_tiles.cu -- serving mode 3: direct-protocol requests as tiles
// of one resident kernel.
//
// The host appends requests to a ring in host-mapped memory.  CTA 0 of the
// kernel (one warp) ingests them in order: it copies each entry into device
// state and publishes it on one of two device queues, small requests and
// large ones.  Every other CTA loops: it claims the next tile (a range of
// 16-byte units) of the first request of the small queue that still has
// tiles, else of the large queue, folds those units exactly as the direct
// protocol's kernels do (each unit's ring chain in the ring schedule's order,
// so the bits are those of a per-call launch with the same plan), and the
// CTA that finishes a request's last tile writes its completion into
// host-mapped memory.  A small request that arrives while a large one runs
// takes the next free CTAs, so it waits for one tile at most, never for the
// large request; large requests share the GPU tile by tile in arrival order.
//
// No CTA waits on another: claims and completions are atomics, and the only
// waits are the idle polls, bounded by the idle timeout and by the stop word.
#include <cuda_runtime.h>

#include <cstddef>

#include "vcomm_direct.cuh"
#include "vcomm_kernels.h"

namespace vc {
namespace {

using namespace direct;

// units per thread per iteration (one body per (dtype, op), out of line, so
// that each keeps its own registers)
template <class T> struct TileNU { static constexpr int value = 2; };
constexpr int kTileThreads = 256;

VDEV uint64_t ldAcquireSys(const unsigned long long* p) {
  uint64_t v;
  asm volatile("ld.acquire.sys.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
VDEV uint64_t ldVol(const unsigned long long* p) { return *(const volatile unsigned long long*)p; }
VDEV void stVol(unsigned long long* p, uint64_t v) { *(volatile unsigned long long*)p = v; }

// 16-byte units read through L2 only: the kernel outlives the requests, and
// a buffer the host rewrote between two requests must not be served from a
// line an SM's L1 kept from the earlier one
template <class T>
struct Unit16L2 {
  using W = uint4;
  static constexpr int kElems = 16 / sizeof(T);
  static VDEV W load(const char* p) { return ldCG(p); }
  static VDEV void store(char* p, W v) { __stcs((uint4*)p, v); }
};
template <class T>
struct Unit1L2 {
  using W = T;
  static constexpr int kElems = 1;
  static VDEV W load(const char* p) {
    if constexpr (sizeof(T) == 1) {
      unsigned short v;
      asm volatile("ld.global.cg.u8 %0, [%1];" : "=h"(v) : "l"(p));
      return (T)v;
    } else if constexpr (std::is_same<T, __half>::value) {
      unsigned short v;
      asm volatile("ld.global.cg.u16 %0, [%1];" : "=h"(v) : "l"(p));
      return __ushort_as_half(v);
    } else if constexpr (std::is_same<T, __nv_bfloat16>::value) {
      unsigned short v;
      asm volatile("ld.global.cg.u16 %0, [%1];" : "=h"(v) : "l"(p));
      return __ushort_as_bfloat16(v);
    } else if constexpr (std::is_same<T, float>::value) {
      unsigned v;
      asm volatile("ld.global.cg.u32 %0, [%1];" : "=r"(v) : "l"(p));
      return __uint_as_float(v);
    } else {
      unsigned v;
      asm volatile("ld.global.cg.u32 %0, [%1];" : "=r"(v) : "l"(p));
      return (T)v;
    }
  }
  static VDEV void store(char* p, W v) { *(T*)p = v; }
};

VDEV DirectView viewOfReq(const ServeReq* q) {
  return DirectView{(const void* const*)q->send, (void* const*)q->recv, q->count, q->chunk, q->inplaceMask,
                    q->coll, q->nranks, q->nsub, q->root, 0};
}

template <class T, class Op>
__device__ __noinline__ void tileReduce(const ServeReq* q, unsigned long long lo, unsigned long long hi,
                                        bool tail) {
  const DirectView v = viewOfReq(q);
  if (q->vec) directReduce<T, Op, Unit16L2<T>, TileNU<T>::value>(v, lo, hi, tail);
  else directReduce<T, Op, Unit1L2<T>, 1>(v, lo, hi, tail);
}

__device__ __noinline__ void tileCopy(const ServeReq* q, unsigned long long lo, unsigned long long hi, bool tail) {
  const DirectView v = viewOfReq(q);
  if (q->vec) directCopy<Unit16L2<uint8_t>>(v, lo, hi, tail);
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

// CTA 0, warp 0: ingest ring entries firstSeq, firstSeq + 1, ... in order
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
      if (ctl->abort) {
        stop = 1;
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

// CTAs 1..: take tiles until the stop word is raised and no tile is left
__device__ void work(const TileArgs& a) {
  __shared__ ServeReq sReq;
  __shared__ long long sSlot;
  __shared__ unsigned long long sTile, sUnits, sTileUnits, sTiles;
  __shared__ int sStop;
  TileQueues* q = a.q;
  unsigned backoff = 64;
  while (true) {
    if (threadIdx.x == 0) {
      long long slot = -1;
      unsigned long long tile = 0;
      for (int c = 0; c < 2 && slot < 0; c++) {
        unsigned long long h = ldVol(&q->head[c]);
        const unsigned long long t = ldAcquire(&q->tail[c]);
        while (h < t) {
          const unsigned long long e = ldVol(&q->entry[c][h % kTileRing]);
          if ((e >> 32) != (h & 0xffffffffull)) break;   // not this position (cannot happen after tail)
          const int s = (int)(e & 0xffffffffull) - 1;
          TileState* st = &a.state[s];
          const unsigned long long tl = atomicAdd(&st->next, 1ull);
          if (tl < ldVol(&st->ntiles)) {
            slot = s;
            tile = tl;
            break;
          }
          atomicCAS(&q->head[c], h, h + 1);               // every tile of entry h is claimed
          h++;
        }
      }
      sStop = (slot < 0 && *(volatile int*)&q->stop) ? 1 : 0;
      sSlot = slot;
      sTile = tile;
      if (slot >= 0) {
        TileState* st = &a.state[slot];
        sUnits = ldVol(&st->units);
        sTileUnits = ldVol(&st->tileUnits);
        sTiles = ldVol(&st->ntiles);
      } else if (!sStop) {
        __nanosleep(backoff);
      }
    }
    __syncthreads();
    if (sStop) return;
    const long long slot = sSlot;
    if (slot < 0) {
      backoff = backoff < 2048 ? 2 * backoff : 2048;
      __syncthreads();   // everyone has read sSlot before thread 0 writes it again
      continue;
    }
    backoff = 64;
    TileState* st = &a.state[slot];
    for (int i = threadIdx.x; i < (int)(sizeof(ServeReq) / 8); i += blockDim.x)
      ((unsigned long long*)&sReq)[i] = ldVol(&((const unsigned long long*)&st->req)[i]);
    __syncthreads();
    const unsigned long long lo = sTile * sTileUnits;
    const unsigned long long hi = lo + sTileUnits < sUnits ? lo + sTileUnits : sUnits;
    runTile(&sReq, lo < hi ? lo : hi, hi, sTile + 1 == sTiles);
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();                                   // this tile's stores before the count
      const unsigned long long d = atomicAdd(&st->done, 1ull);
      if (d + 1 == sTiles) {                             // the request's last tile: report it
        __threadfence();
        TileDone* dn = &a.done[slot];
        stVol(&dn->tStart, ldVol(&st->tStart));
        stVol(&dn->tEnd, globaltimer());
        __threadfence_system();
        stVol(&dn->seq, ldVol(&st->seq));
        __threadfence_system();
        atomicAdd(&q->completed, 1ull);
      }
    }
    __syncthreads();   // sReq and the shared words are free again
  }
}

__global__ void __launch_bounds__(kTileThreads, 1) kServeTiles(const __grid_constant__ TileArgs a) {
  if (blockIdx.x == 0) {
    if (threadIdx.x < 32) ingest(a);
    return;
  }
  work(a);
}

}  // namespace

const void* serveTilesKernel() { return (const void*)kServeTiles; }
int serveTilesThreads() { return kTileThreads; }
int serveTilesUnitsPerIter() { return kTileThreads * 2; }

}  // namespace vc
