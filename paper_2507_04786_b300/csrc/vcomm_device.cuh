// vcomm_device.cuh -- device side of the virtual-rank collectives (sm_103a).
//
// One CTA (or one warp group of a CTA) is the worker of one (vrank, channel).
// Workers exchange data only through connection FIFOs in HBM.  The three
// protocols of Sec. III differ in how a FIFO slot is filled and signalled:
//   Simple : plain 16-byte stores into the slot, a gpu-scope fence, then a
//            release store of the connection's `tail` counter; the receiver
//            acquires `tail` before it reads the slot (Sec. III-A).
//   LL     : 8-byte lines {4 data bytes, 4-byte flag} written with one 8-byte
//            store each; the reader polls the flag of every line (Sec. III-B).
//   LL128  : 128-byte lines of 120 data bytes + an 8-byte flag, written by 8
//            threads in one warp-wide 16-byte store instruction; the reader
//            loads the whole line and checks the flag (Sec. III-C).
// All three return a slot to the sender with a release store of `head`
// (credits), so the FIFO holds at most `nsteps` steps in flight (Sec. V-C).
// Every wait is bounded by %globaltimer; on expiry (or on the host abort word)
// the worker records the failure and returns -- no trap, no endless loop.
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include "vcomm_internal.h"

namespace vc {

#define VDEV __device__ __forceinline__

// ------------------------------------------------------------------ PTX helpers
VDEV uint64_t globaltimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
VDEV uint64_t ldAcquire(const unsigned long long* p) {
  uint64_t v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
VDEV void stRelease(unsigned long long* p, uint64_t v) {
  asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
VDEV void stRelaxed(unsigned long long* p, uint64_t v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
VDEV void ldVolatile2(const void* p, uint64_t& a, uint64_t& b) {
  asm volatile("ld.volatile.global.v2.u64 {%0, %1}, [%2];" : "=l"(a), "=l"(b) : "l"(p) : "memory");
}
VDEV void stVolatile2(void* p, uint64_t a, uint64_t b) {
  asm volatile("st.volatile.global.v2.u64 [%0], {%1, %2};" ::"l"(p), "l"(a), "l"(b) : "memory");
}
// 16-byte loads that bypass L1 (FIFO slots are rewritten by other SMs)
VDEV uint4 ldCG(const void* p) {
  uint4 v;
  asm volatile("ld.global.cg.v4.u32 {%0, %1, %2, %3}, [%4];"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "l"(p));
  return v;
}
VDEV void st16(void* p, uint4 v) {
  asm volatile("st.global.v4.u32 [%0], {%1, %2, %3, %4};" ::"l"(p), "r"(v.x), "r"(v.y), "r"(v.z),
               "r"(v.w) : "memory");
}
VDEV void groupBar(int id, int nthreads) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

// ------------------------------------------------------------------ element ops
// f(a, b): a is the received operand, b the local one.  Sums are IEEE
// round-to-nearest-even in the element type (16-bit types widen to fp32 and
// round once, which equals the correctly rounded 16-bit sum); max keeps the
// received operand on ties.
struct OpSum {};
struct OpMax {};
struct OpNone {};

template <class T, class Op> struct ElemOp;
template <> struct ElemOp<float, OpSum> {
  static VDEV float f(float a, float b) { return __fadd_rn(a, b); }
};
template <> struct ElemOp<float, OpMax> {
  static VDEV float f(float a, float b) { return (b > a) ? b : a; }
};
template <> struct ElemOp<int32_t, OpSum> {
  static VDEV int32_t f(int32_t a, int32_t b) { return (int32_t)((uint32_t)a + (uint32_t)b); }
};
template <> struct ElemOp<int32_t, OpMax> {
  static VDEV int32_t f(int32_t a, int32_t b) { return (b > a) ? b : a; }
};
template <> struct ElemOp<__half, OpSum> {
  static VDEV __half f(__half a, __half b) {
    return __float2half_rn(__fadd_rn(__half2float(a), __half2float(b)));
  }
};
template <> struct ElemOp<__half, OpMax> {
  static VDEV __half f(__half a, __half b) { return (__half2float(b) > __half2float(a)) ? b : a; }
};
template <> struct ElemOp<__nv_bfloat16, OpSum> {
  static VDEV __nv_bfloat16 f(__nv_bfloat16 a, __nv_bfloat16 b) {
    return __float2bfloat16_rn(__fadd_rn(__bfloat162float(a), __bfloat162float(b)));
  }
};
template <> struct ElemOp<__nv_bfloat16, OpMax> {
  static VDEV __nv_bfloat16 f(__nv_bfloat16 a, __nv_bfloat16 b) {
    return (__bfloat162float(b) > __bfloat162float(a)) ? b : a;
  }
};
template <class T> struct ElemOp<T, OpNone> {
  static VDEV T f(T a, T) { return a; }
};

// apply f lane-wise on raw words (W = uint4 or uint64_t)
template <class T, class Op, class W>
VDEV W applyWord(W a, W b) {
  constexpr int n = sizeof(W) / sizeof(T);
  union U { W w; T e[n]; };
  U ua, ub, uo;
  ua.w = a;
  ub.w = b;
#pragma unroll
  for (int i = 0; i < n; i++) uo.e[i] = ElemOp<T, Op>::f(ua.e[i], ub.e[i]);
  return uo.w;
}

// ------------------------------------------------------------------ failure handling
VDEV void reportFailure(const KernArgs& a, int code, int rank, int ch, int where) {
  if (atomicCAS(a.errClaim, 0, code) == 0) {
    volatile ErrWord* e = a.err;
    e->rank = rank;
    e->channel = ch;
    e->where = where;
    __threadfence_system();
    e->code = code;
    __threadfence_system();
  }
}

// Spin until *p >= v.  Returns false (after recording why) on deadline or abort.
VDEV bool waitGeq(const KernArgs& a, const unsigned long long* p, uint64_t v, int rank, int ch,
                  int where) {
  if (ldAcquire(p) >= v) return true;
  uint64_t t0 = globaltimer();
  unsigned it = 0;
  while (true) {
    if (ldAcquire(p) >= v) return true;
    if (((++it) & 127u) == 0) {
      if (*a.abortFlag) { reportFailure(a, vAborted, rank, ch, where); return false; }
      if (globaltimer() - t0 > a.timeoutNs) { reportFailure(a, vTimeout, rank, ch, where); return false; }
    }
  }
}

// ------------------------------------------------------------------ user-memory words
// Load `valid` (<= 8) bytes at p as one little-endian word, zero padded.  Fast
// path: p 8-byte aligned and a full word.  Slow path: element-wise loads of
// the element size (pointers are always element aligned).
template <class T>
VDEV uint64_t loadUser8(const char* p, int valid) {
  if (valid <= 0) return 0;
  if (valid == 8 && (((uintptr_t)p) & 7) == 0) return *(const uint64_t*)p;
  uint64_t v = 0;
  for (int b = 0; b < valid; b += (int)sizeof(T)) {
    uint64_t e;
    if (sizeof(T) == 4) e = *(const uint32_t*)(p + b);
    else if (sizeof(T) == 2) e = *(const uint16_t*)(p + b);
    else e = *(const uint8_t*)(p + b);
    v |= e << (8 * b);
  }
  return v;
}
template <class T>
VDEV void storeUser8(char* p, uint64_t v, int valid) {
  if (valid <= 0) return;
  if (valid == 8 && (((uintptr_t)p) & 7) == 0) { *(uint64_t*)p = v; return; }
  for (int b = 0; b < valid; b += (int)sizeof(T)) {
    uint64_t e = v >> (8 * b);
    if (sizeof(T) == 4) *(uint32_t*)(p + b) = (uint32_t)e;
    else if (sizeof(T) == 2) *(uint16_t*)(p + b) = (uint16_t)e;
    else *(uint8_t*)(p + b) = (uint8_t)e;
  }
}

// ------------------------------------------------------------------ Simple reduce-copy
// d*[i] = fold over the NSRC sources: v = s0[i]; v = f(s1[i], v); v = f(s2[i], v).
// 16-byte vectors with UNROLL packs per thread in flight; element-wise tail,
// and an element-wise path when any pointer is not 16-byte aligned.
template <class T, class Op, int NSRC>
__device__ __noinline__ void reduceCopy(int tid, int nthr, const char* s0, const char* s1,
                                        const char* s2, char* d0, char* d1, char* d2, int nd,
                                        unsigned long long nbytes) {
  constexpr int UNROLL = (NSRC >= 3) ? 2 : 4;
  uintptr_t orall = (uintptr_t)s0 | (uintptr_t)d0;
  if (NSRC > 1) orall |= (uintptr_t)s1;
  if (NSRC > 2) orall |= (uintptr_t)s2;
  if (nd > 1) orall |= (uintptr_t)d1;
  if (nd > 2) orall |= (uintptr_t)d2;
  unsigned long long done = 0;
  if ((orall & 15) == 0) {
    const unsigned long long npk = nbytes / 16;
    const uint4* a4 = (const uint4*)s0;
    const uint4* b4 = (const uint4*)s1;
    const uint4* c4 = (const uint4*)s2;
    for (unsigned long long p0 = tid; p0 < npk; p0 += (unsigned long long)UNROLL * nthr) {
      uint4 v[UNROLL], w1[UNROLL], w2[UNROLL];
#pragma unroll
      for (int u = 0; u < UNROLL; u++) {
        const unsigned long long i = p0 + (unsigned long long)u * nthr;
        if (i < npk) {
          v[u] = ldCG(a4 + i);
          if (NSRC > 1) w1[u] = ldCG(b4 + i);
          if (NSRC > 2) w2[u] = ldCG(c4 + i);
        }
      }
#pragma unroll
      for (int u = 0; u < UNROLL; u++) {
        const unsigned long long i = p0 + (unsigned long long)u * nthr;
        if (i < npk) {
          if (NSRC > 1) v[u] = applyWord<T, Op>(w1[u], v[u]);
          if (NSRC > 2) v[u] = applyWord<T, Op>(w2[u], v[u]);
          st16((uint4*)d0 + i, v[u]);
          if (nd > 1) st16((uint4*)d1 + i, v[u]);
          if (nd > 2) st16((uint4*)d2 + i, v[u]);
        }
      }
    }
    done = npk * 16;
  }
  // element-wise remainder (or everything when misaligned)
  const unsigned long long ne = (nbytes - done) / sizeof(T);
  for (unsigned long long e = tid; e < ne; e += nthr) {
    const unsigned long long off = done + e * sizeof(T);
    T v = *(const T*)(s0 + off);
    if (NSRC > 1) v = ElemOp<T, Op>::f(*(const T*)(s1 + off), v);
    if (NSRC > 2) v = ElemOp<T, Op>::f(*(const T*)(s2 + off), v);
    *(T*)(d0 + off) = v;
    if (nd > 1) *(T*)(d1 + off) = v;
    if (nd > 2) *(T*)(d2 + off) = v;
  }
}

// ------------------------------------------------------------------ LL / LL128 line codecs
// LL: line pair p (16 bytes) carries data bytes [8p, 8p+8): line 2p holds
// bytes 8p..8p+3 in its low word, line 2p+1 bytes 8p+4..8p+7; every line's
// high word is the 32-bit flag.
VDEV void llStorePair(char* slot, unsigned long long p, uint64_t v, uint32_t flag) {
  uint64_t f = (uint64_t)flag << 32;
  stVolatile2(slot + 16 * p, (v & 0xffffffffull) | f, (v >> 32) | f);
}
// poll pair p until both lines carry `flag`; false on deadline / abort
VDEV bool llLoadPair(const KernArgs& a, const char* slot, unsigned long long p, uint32_t flag,
                     uint64_t& v, volatile int* sAbort, int rank, int ch) {
  uint64_t x, y;
  unsigned it = 0;
  uint64_t t0 = 0;
  while (true) {
    ldVolatile2(slot + 16 * p, x, y);
    if ((uint32_t)(x >> 32) == flag && (uint32_t)(y >> 32) == flag) break;
    if (((++it) & 255u) == 0) {
      if (*sAbort) return false;
      if (*a.abortFlag) { reportFailure(a, vAborted, rank, ch, 3); *sAbort = 1; return false; }
      uint64_t now = globaltimer();
      if (t0 == 0) t0 = now;
      else if (now - t0 > a.timeoutNs) { reportFailure(a, vTimeout, rank, ch, 3); *sAbort = 1; return false; }
    }
  }
  v = (x & 0xffffffffull) | (y << 32);
  return true;
}

// LL128: line L (128 bytes) carries data bytes [120 L, 120 L + 120) in words
// 0..14 and the 64-bit flag in word 15.  Thread j (0..7) of the line's 8-lane
// group holds words 2j and 2j+1; lane 7 holds word 14 (data) and the flag.
VDEV void ll128Store(char* slot, unsigned long long line, int j, uint64_t v0, uint64_t v1,
                     uint64_t flag) {
  stVolatile2(slot + 128 * line + 16 * j, v0, j == 7 ? flag : v1);
}
// warp-collective: every lane of the warp calls it; lanes of lines beyond the
// data pass lineValid = false.  Returns false on deadline / abort (warp-uniform).
VDEV bool ll128Load(const KernArgs& a, const char* slot, unsigned long long line, int lane,
                    bool lineValid, uint64_t flag, uint64_t& v0, uint64_t& v1,
                    volatile int* sAbort, int rank, int ch) {
  const int j = lane & 7;
  unsigned it = 0;
  uint64_t t0 = 0;
  v0 = 0;
  v1 = 0;
  while (true) {
    if (lineValid) ldVolatile2(slot + 128 * line + 16 * j, v0, v1);
    bool mine = !lineValid || j != 7 || v1 == flag;
    bool lineOk = __shfl_sync(0xffffffffu, mine, lane | 7);
    if (__all_sync(0xffffffffu, lineOk)) return true;
    if (((++it) & 255u) == 0) {
      int stop = 0;
      if (lane == 0) {
        if (*sAbort) stop = 1;
        else if (*a.abortFlag) { reportFailure(a, vAborted, rank, ch, 3); *sAbort = 1; stop = 1; }
        else {
          uint64_t now = globaltimer();
          if (t0 == 0) t0 = now;
          else if (now - t0 > a.timeoutNs) { reportFailure(a, vTimeout, rank, ch, 3); *sAbort = 1; stop = 1; }
        }
      }
      if (__shfl_sync(0xffffffffu, stop, 0)) return false;
    }
  }
}

// ------------------------------------------------------------------ primitives
// A Prims object is one worker's view of its connections: up to two receive
// connections (all read by a recv* primitive) and up to two send connections
// (all written by a *send primitive).  The seven primitives of Sec. V-B are
// the combinations of (receive?, local input?, send?, user output?).
template <int PROTO, class T, class Op>
struct Prims {
  const KernArgs& a;
  int tid, nthr, barId;
  volatile int* sAbort;
  int rank, ch;
  const ConnDev* rc[2];
  const ConnDev* sc[2];
  int nrc, nsc;
  uint64_t rstep[2], sstep[2];

  VDEV Prims(const KernArgs& args, int tid_, int nthr_, int barId_, volatile int* sAbort_, int rank_,
             int ch_, const ConnDev* r0, const ConnDev* r1, const ConnDev* s0, const ConnDev* s1)
      : a(args), tid(tid_), nthr(nthr_), barId(barId_), sAbort(sAbort_), rank(rank_), ch(ch_) {
    nrc = 0;
    nsc = 0;
    if (r0) rc[nrc++] = r0;
    if (r1) rc[nrc++] = r1;
    if (s0) sc[nsc++] = s0;
    if (s1) sc[nsc++] = s1;
    // the step counters: a worker is the only writer of its send conns' tail
    // and its receive conns' head, so their current values are its position
    for (int i = 0; i < nrc; i++) rstep[i] = ldAcquire(rc[i]->head);
    for (int i = 0; i < nsc; i++) sstep[i] = ldAcquire(sc[i]->tail);
  }

  VDEV void bar() { groupBar(barId, nthr); }
  VDEV char* slotOf(const ConnDev* c, uint64_t step) const {
    return c->buf + (step % (uint64_t)a.nsteps) * a.slotBytes;
  }

  // wait for data (Simple only) and for send credits, then a group barrier
  VDEV bool acquire(bool doRecv, bool doSend) {
    if (tid == 0) {
      bool ok = true;
      if (PROTO == kSimple && doRecv)
        for (int i = 0; i < nrc && ok; i++) ok = waitGeq(a, rc[i]->tail, rstep[i] + 1, rank, ch, 1);
      if (doSend)
        for (int i = 0; i < nsc && ok; i++)
          if (sstep[i] + 1 > (uint64_t)a.nsteps)
            ok = waitGeq(a, sc[i]->head, sstep[i] + 1 - (uint64_t)a.nsteps, rank, ch, 2);
      if (!ok) *sAbort = 1;
    }
    bar();
    return *sAbort == 0;
  }

  // publish the step: tail for sends, head for receives
  VDEV bool release(bool doRecv, bool doSend) {
    if (PROTO == kSimple) __threadfence();
    bar();
    if (*sAbort) return false;
    if (tid == 0) {
      if (doSend)
        for (int i = 0; i < nsc; i++) {
          if (PROTO == kSimple) stRelease(sc[i]->tail, sstep[i] + 1);
          else stRelaxed(sc[i]->tail, sstep[i] + 1);
        }
      if (doRecv)
        for (int i = 0; i < nrc; i++) stRelease(rc[i]->head, rstep[i] + 1);
    }
    if (doSend)
      for (int i = 0; i < nsc; i++) sstep[i]++;
    if (doRecv)
      for (int i = 0; i < nrc; i++) rstep[i]++;
    return true;
  }

  // one FIFO step of m units (m <= slotUnits); out of line to keep the
  // collectives' code small
  __device__ __noinline__ bool step(bool doRecv, bool doLocal, bool doSend, bool doOut, const T* local, T* out,
                 unsigned long long m) {
    if (!acquire(doRecv, doSend)) return false;
    const unsigned long long nbytes = m * sizeof(T);
    if (PROTO == kSimple) {
      const char* src[3] = {nullptr, nullptr, nullptr};
      char* dst[3] = {nullptr, nullptr, nullptr};
      int ns = 0, nd = 0;
      if (doLocal) src[ns++] = (const char*)local;
      if (doRecv)
        for (int i = 0; i < nrc; i++) src[ns++] = slotOf(rc[i], rstep[i]);
      if (doOut) dst[nd++] = (char*)out;
      if (doSend)
        for (int i = 0; i < nsc; i++) dst[nd++] = slotOf(sc[i], sstep[i]);
      if (ns == 1) reduceCopy<T, Op, 1>(tid, nthr, src[0], src[1], src[2], dst[0], dst[1], dst[2], nd, nbytes);
      else if (ns == 2) reduceCopy<T, Op, 2>(tid, nthr, src[0], src[1], src[2], dst[0], dst[1], dst[2], nd, nbytes);
      else reduceCopy<T, Op, 3>(tid, nthr, src[0], src[1], src[2], dst[0], dst[1], dst[2], nd, nbytes);
    } else if (PROTO == kLL) {
      const unsigned long long npairs = (nbytes + 7) / 8;
      const char* rs[2];
      char* ss[2];
      uint32_t rf[2];
      uint32_t sf[2];
      for (int i = 0; i < nrc; i++) { rs[i] = slotOf(rc[i], rstep[i]); rf[i] = (uint32_t)(rstep[i] + 1); }
      for (int i = 0; i < nsc; i++) { ss[i] = slotOf(sc[i], sstep[i]); sf[i] = (uint32_t)(sstep[i] + 1); }
      for (unsigned long long p = tid; p < npairs; p += nthr) {
        const int valid = (int)((nbytes - 8 * p) < 8 ? (nbytes - 8 * p) : 8);
        uint64_t v = 0;
        int first = 0;
        if (doLocal) {
          v = loadUser8<T>((const char*)local + 8 * p, valid);
        } else {
          if (!llLoadPair(a, rs[0], p, rf[0], v, sAbort, rank, ch)) break;
          first = 1;
        }
        bool fail = false;
        if (doRecv)
          for (int i = first; i < nrc; i++) {
            uint64_t w;
            if (!llLoadPair(a, rs[i], p, rf[i], w, sAbort, rank, ch)) { fail = true; break; }
            v = applyWord<T, Op>(w, v);
          }
        if (fail) break;
        if (doOut) storeUser8<T>((char*)out + 8 * p, v, valid);
        if (doSend)
          for (int i = 0; i < nsc; i++) llStorePair(ss[i], p, v, sf[i]);
      }
    } else {  // LL128
      const unsigned long long nlines = (nbytes + 119) / 120;
      const unsigned long long nquads = (nlines + 3) / 4;
      const int warp = tid >> 5, lane = tid & 31, nwarps = nthr >> 5;
      const int j = lane & 7;
      const char* rs[2];
      char* ss[2];
      uint64_t rf[2], sf[2];
      for (int i = 0; i < nrc; i++) { rs[i] = slotOf(rc[i], rstep[i]); rf[i] = rstep[i] + 1; }
      for (int i = 0; i < nsc; i++) { ss[i] = slotOf(sc[i], sstep[i]); sf[i] = sstep[i] + 1; }
      for (unsigned long long q = warp; q < nquads; q += nwarps) {
        const unsigned long long line = 4 * q + (lane >> 3);
        const bool lineValid = line < nlines;
        const unsigned long long uoff = 120 * line + 16 * (unsigned long long)j;
        const int cap = (j == 7) ? 8 : 16;
        long long rem = lineValid ? (long long)nbytes - (long long)uoff : 0;
        const int valid = rem <= 0 ? 0 : (rem < cap ? (int)rem : cap);
        const int valid0 = valid < 8 ? valid : 8;
        const int valid1 = valid > 8 ? valid - 8 : 0;
        uint64_t v0 = 0, v1 = 0;
        int first = 0;
        bool fail = false;
        if (doLocal) {
          v0 = loadUser8<T>((const char*)local + uoff, valid0);
          v1 = loadUser8<T>((const char*)local + uoff + 8, valid1);
        } else {
          if (!ll128Load(a, rs[0], line, lane, lineValid, rf[0], v0, v1, sAbort, rank, ch)) fail = true;
          first = 1;
        }
        if (!fail && doRecv)
          for (int i = first; i < nrc; i++) {
            uint64_t w0, w1;
            if (!ll128Load(a, rs[i], line, lane, lineValid, rf[i], w0, w1, sAbort, rank, ch)) {
              fail = true;
              break;
            }
            v0 = applyWord<T, Op>(w0, v0);
            v1 = applyWord<T, Op>(w1, v1);
          }
        if (fail) break;   // warp-uniform
        if (doOut && valid > 0) {
          storeUser8<T>((char*)out + uoff, v0, valid0);
          storeUser8<T>((char*)out + uoff + 8, v1, valid1);
        }
        if (doSend && lineValid)
          for (int i = 0; i < nsc; i++) ll128Store(ss[i], line, j, v0, v1, sf[i]);
      }
    }
    return release(doRecv, doSend);
  }

  // a primitive over n units, in FIFO steps of at most slotUnits
  VDEV bool run(bool doRecv, bool doLocal, bool doSend, bool doOut, const T* local, T* out,
                unsigned long long n) {
    unsigned long long done = 0;
    while (done < n) {
      unsigned long long m = n - done;
      if (m > a.slotUnits) m = a.slotUnits;
      if (!step(doRecv, doLocal, doSend, doOut, local ? local + done : nullptr,
                out ? out + done : nullptr, m))
        return false;
      done += m;
    }
    return true;
  }

  // Sec. V-B primitive names
  VDEV bool send(const T* x, unsigned long long n) { return run(false, true, true, false, x, nullptr, n); }
  VDEV bool recv(T* y, unsigned long long n) { return run(true, false, false, true, nullptr, y, n); }
  VDEV bool recvReduceSend(const T* x, unsigned long long n) { return run(true, true, true, false, x, nullptr, n); }
  VDEV bool recvCopySend(T* y, unsigned long long n) { return run(true, false, true, true, nullptr, y, n); }
  VDEV bool recvReduceCopySend(const T* x, T* y, unsigned long long n) { return run(true, true, true, true, x, y, n); }
  VDEV bool copySend(const T* x, T* y, unsigned long long n) { return run(false, true, true, true, x, y, n); }
  VDEV bool recvReduceCopy(const T* x, T* y, unsigned long long n) { return run(true, true, false, true, x, y, n); }
};

// ------------------------------------------------------------------ collectives
// Ring AllReduce, Table "Steps in one loop iteration of NCCL Ring AllReduce":
// at step t rank r handles segment (r - t - 1) mod k of the loop.
template <int P, class T, class Op>
VDEV void ringAllReduce(const KernArgs& a, int r, int ch, volatile int* sAbort) {
  const int k = a.nranks;
  const ConnDev* sc = &a.conns[ch * k + r];
  const ConnDev* rc = &a.conns[ch * k + modk(r - 1, k)];
  Prims<P, T, Op> pr(a, threadIdx.x, blockDim.x, 0, sAbort, r, ch, rc, nullptr, sc, nullptr);
  unsigned long long start, len;
  channelRange(a.count, sizeof(T), a.nsub, ch, &start, &len);
  const unsigned long long end = start + len, loop = (unsigned long long)k * a.chunk;
  const T* x = (const T*)a.send[r];
  T* y = (T*)a.recv[r];
  for (unsigned long long off = start; off < end; off += loop) {
    const unsigned long long c = ringLoopChunk(off, end, k, a.chunk, sizeof(T));
    for (int t = 0; t <= 2 * k - 2; t++) {
      const int s = modk(r - t - 1, k);
      unsigned long long sa = off + (unsigned long long)s * c;
      if (sa > end) sa = end;
      unsigned long long sb = sa + c;
      if (sb > end) sb = end;
      const unsigned long long n = sb - sa;
      bool ok;
      if (t == 0) ok = pr.send(x + sa, n);
      else if (t <= k - 2) ok = pr.recvReduceSend(x + sa, n);
      else if (t == k - 1) ok = pr.recvReduceCopySend(x + sa, y + sa, n);
      else if (t <= 2 * k - 3) ok = pr.recvCopySend(y + sa, n);
      else ok = pr.recv(y + sa, n);
      if (!ok) return;
    }
  }
}

// Ring ReduceScatter, Table "Steps in one loop iteration of NCCL Ring ReduceScatter"
template <int P, class T, class Op>
VDEV void ringReduceScatter(const KernArgs& a, int r, int ch, volatile int* sAbort) {
  const int k = a.nranks;
  const ConnDev* sc = &a.conns[ch * k + r];
  const ConnDev* rc = &a.conns[ch * k + modk(r - 1, k)];
  Prims<P, T, Op> pr(a, threadIdx.x, blockDim.x, 0, sAbort, r, ch, rc, nullptr, sc, nullptr);
  unsigned long long start, len;
  channelRange(a.count, sizeof(T), a.nsub, ch, &start, &len);
  const unsigned long long end = start + len;
  const T* x = (const T*)a.send[r];
  T* y = (T*)a.recv[r];
  for (unsigned long long off = start; off < end; off += a.chunk) {
    const unsigned long long n = (end - off < a.chunk) ? end - off : a.chunk;
    for (int t = 0; t <= k - 1; t++) {
      const int s = modk(r - t - 1, k);
      const T* src = x + (unsigned long long)s * a.count + off;
      bool ok;
      if (t == 0) ok = pr.send(src, n);
      else if (t <= k - 2) ok = pr.recvReduceSend(src, n);
      else ok = pr.recvReduceCopy(src, y + off, n);
      if (!ok) return;
    }
  }
}

// Ring AllGather, Table "Steps in one loop iteration of NCCL Ring AllGather";
// units are bytes (Sec. V-C), a.count = bytes per rank
template <int P>
VDEV void ringAllGather(const KernArgs& a, int r, int ch, volatile int* sAbort) {
  using T = uint8_t;
  const int k = a.nranks;
  const ConnDev* sc = &a.conns[ch * k + r];
  const ConnDev* rc = &a.conns[ch * k + modk(r - 1, k)];
  Prims<P, T, OpNone> pr(a, threadIdx.x, blockDim.x, 0, sAbort, r, ch, rc, nullptr, sc, nullptr);
  unsigned long long start, len;
  channelRange(a.count, 1, a.nsub, ch, &start, &len);
  const unsigned long long end = start + len;
  const T* x = (const T*)a.send[r];
  T* y = (T*)a.recv[r];
  for (unsigned long long off = start; off < end; off += a.chunk) {
    const unsigned long long n = (end - off < a.chunk) ? end - off : a.chunk;
    for (int t = 0; t <= k - 1; t++) {
      T* dst = y + (unsigned long long)modk(r - t, k) * a.count + off;
      bool ok;
      if (t == 0) ok = ((a.inplaceMask >> r) & 1) ? pr.send(dst, n) : pr.copySend(x + off, dst, n);
      else if (t <= k - 2) ok = pr.recvCopySend(dst, n);
      else ok = pr.recv(dst, n);
      if (!ok) return;
    }
  }
}

// Ring Broadcast chain root -> root+1 -> ... (Table "Ring Broadcast"), bytes
template <int P>
VDEV void ringBroadcast(const KernArgs& a, int r, int ch, volatile int* sAbort) {
  using T = uint8_t;
  const int k = a.nranks;
  const int pos = modk(r - a.root, k);
  const ConnDev* sc = (pos < k - 1) ? &a.conns[ch * k + r] : nullptr;
  const ConnDev* rc = (pos > 0) ? &a.conns[ch * k + modk(r - 1, k)] : nullptr;
  Prims<P, T, OpNone> pr(a, threadIdx.x, blockDim.x, 0, sAbort, r, ch, rc, nullptr, sc, nullptr);
  unsigned long long start, len;
  channelRange(a.count, 1, a.nsub, ch, &start, &len);
  const unsigned long long end = start + len;
  const T* x = (const T*)a.send[r];
  T* y = (T*)a.recv[r];
  for (unsigned long long off = start; off < end; off += a.chunk) {
    const unsigned long long n = (end - off < a.chunk) ? end - off : a.chunk;
    bool ok;
    if (pos == 0) ok = ((a.inplaceMask >> r) & 1) ? pr.send(x + off, n) : pr.copySend(x + off, y + off, n);
    else if (pos < k - 1) ok = pr.recvCopySend(y + off, n);
    else ok = pr.recv(y + off, n);
    if (!ok) return;
  }
}

// Ring Reduce chain root+1 -> ... -> root (Table "Ring Reduce")
template <int P, class T, class Op>
VDEV void ringReduce(const KernArgs& a, int r, int ch, volatile int* sAbort) {
  const int k = a.nranks;
  const int pos = modk(r - a.root - 1, k);
  const ConnDev* sc = (pos < k - 1) ? &a.conns[ch * k + r] : nullptr;
  const ConnDev* rc = (pos > 0) ? &a.conns[ch * k + modk(r - 1, k)] : nullptr;
  Prims<P, T, Op> pr(a, threadIdx.x, blockDim.x, 0, sAbort, r, ch, rc, nullptr, sc, nullptr);
  unsigned long long start, len;
  channelRange(a.count, sizeof(T), a.nsub, ch, &start, &len);
  const unsigned long long end = start + len;
  const T* x = (const T*)a.send[r];
  T* y = (T*)a.recv[r];
  for (unsigned long long off = start; off < end; off += a.chunk) {
    const unsigned long long n = (end - off < a.chunk) ? end - off : a.chunk;
    bool ok;
    if (pos == 0) ok = pr.send(x + off, n);
    else if (pos < k - 1) ok = pr.recvReduceSend(x + off, n);
    else ok = pr.recvReduceCopy(x + off, y + off, n);
    if (!ok) return;
  }
}

// Tree AllReduce on the double binary tree (Sec. II-C, Table "Steps in one
// loop iteration of NCCL Tree AllReduce").  Sub-channel j runs tree j % 2 on
// its own range.  A non-root worker splits its threads into a reduce group
// (recvReduceSend / send towards the root) and a broadcast group
// (recvCopySend / recv from the root), so both phases stream concurrently;
// the root runs recvReduceCopySend with all its threads.
template <int P, class T, class Op>
VDEV void treeAllReduce(const KernArgs& a, int r, int j, volatile int* sAbort) {
  const int k = a.nranks;
  const int t = j & 1;
  int parent, c0, c1;
  treeLinks(k, t, r, &parent, &c0, &c1);
  const ConnDev* up = a.conns;                                  // [j * k + rank]: rank -> parent
  const ConnDev* down = a.conns + a.downOffset;                  // [j * k + rank]: parent -> rank
  const ConnDev* upC0 = c0 >= 0 ? &up[j * k + c0] : nullptr;
  const ConnDev* upC1 = c1 >= 0 ? &up[j * k + c1] : nullptr;
  const ConnDev* dnC0 = c0 >= 0 ? &down[j * k + c0] : nullptr;
  const ConnDev* dnC1 = c1 >= 0 ? &down[j * k + c1] : nullptr;
  unsigned long long start, len;
  channelRange(a.count, sizeof(T), a.nsub, j, &start, &len);
  const unsigned long long end = start + len;
  const T* x = (const T*)a.send[r];
  T* y = (T*)a.recv[r];
  if (parent < 0) {
    Prims<P, T, Op> pr(a, threadIdx.x, blockDim.x, 0, sAbort, r, j, upC0, upC1, dnC0, dnC1);
    for (unsigned long long off = start; off < end; off += a.chunk) {
      const unsigned long long n = (end - off < a.chunk) ? end - off : a.chunk;
      if (!pr.recvReduceCopySend(x + off, y + off, n)) return;
    }
    return;
  }
  const int nUp = a.upThreads;
  const bool isUp = (int)threadIdx.x < nUp;
  const int gtid = isUp ? threadIdx.x : threadIdx.x - nUp;
  const int gn = isUp ? nUp : (int)blockDim.x - nUp;
  volatile int* gAbort = sAbort + (isUp ? 0 : 1);
  if (isUp) {
    Prims<P, T, Op> pr(a, gtid, gn, 1, gAbort, r, j, upC0, upC1, &up[j * k + r], nullptr);
    const bool leaf = (c0 < 0);
    for (unsigned long long off = start; off < end; off += a.chunk) {
      const unsigned long long n = (end - off < a.chunk) ? end - off : a.chunk;
      if (!(leaf ? pr.send(x + off, n) : pr.recvReduceSend(x + off, n))) return;
    }
  } else {
    Prims<P, T, Op> pr(a, gtid, gn, 2, gAbort, r, j, &down[j * k + r], nullptr, dnC0, dnC1);
    const bool leaf = (c0 < 0);
    for (unsigned long long off = start; off < end; off += a.chunk) {
      const unsigned long long n = (end - off < a.chunk) ? end - off : a.chunk;
      if (!(leaf ? pr.recv(y + off, n) : pr.recvCopySend(y + off, n))) return;
    }
  }
}

// single-rank communicator: every collective is a copy of the local range
template <class T>
VDEV void localCopy(const KernArgs& a, int ch) {
  unsigned long long start, len;
  channelRange(a.count, sizeof(T), a.nsub, ch, &start, &len);
  if ((a.inplaceMask & 1) || len == 0) return;
  reduceCopy<T, OpNone, 1>(threadIdx.x, blockDim.x, (const char*)((const T*)a.send[0] + start),
                           nullptr, nullptr, (char*)((T*)a.recv[0] + start), nullptr, nullptr, 1,
                           len * sizeof(T));
}

}  // namespace vc
