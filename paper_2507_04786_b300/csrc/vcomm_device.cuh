// vcomm_device.cuh -- device side of the virtual-rank collectives (sm_103a).
//
// One CTA (or one warp group of a CTA) is the worker of one (vrank, channel).
// Workers exchange data only through connection FIFOs in HBM.  The three
// protocols of Sec. III differ in how a FIFO slot is filled and signalled:
//   Simple : plain 16-byte stores into the slot, the block barrier, then one
//            thread's gpu-scope release fence and store of the connection's
//            `tail` counter; the receiver acquires `tail` before it reads the
//            slot (Sec. III-A).
//   LL     : 8-byte lines {4 data bytes, 4-byte flag} written with one 8-byte
//            store each; the reader polls the flag of every line (Sec. III-B).
//   LL128  : 128-byte lines of 120 data bytes + an 8-byte flag, written by 8
//            threads in one warp-wide 16-byte store instruction; the reader
//            loads the whole line and checks the flag (Sec. III-C).
// All three return a slot to the sender by advancing `head` (credits: after a
// release fence for Simple, a relaxed store for LL / LL128, whose data the
// flags publish), so the FIFO holds at most `nsteps` steps in flight (Sec. V-C).
// Every wait is bounded by %globaltimer; on expiry (or on the host abort word)
// the worker records the failure and returns -- no trap, no endless loop.
#pragma once
#include <type_traits>
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
VDEV void fenceAcqRel() { asm volatile("fence.acq_rel.gpu;" ::: "memory"); }
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
struct OpProd {};
struct OpMin {};
struct OpAvg {};   // adds like OpSum; the completing step divides by KernArgs::postDiv
struct OpNone {};

// element type of each dtype code (the order of vDataType_t)
template <int D> struct DTypeOf;
template <> struct DTypeOf<kI32> { using T = int32_t; };
template <> struct DTypeOf<kF32> { using T = float; };
template <> struct DTypeOf<kF16> { using T = __half; };
template <> struct DTypeOf<kBF16> { using T = __nv_bfloat16; };
template <> struct DTypeOf<kI8> { using T = int8_t; };
template <> struct DTypeOf<kU8> { using T = uint8_t; };
template <> struct DTypeOf<kU32> { using T = uint32_t; };
template <> struct DTypeOf<kI64> { using T = int64_t; };
template <> struct DTypeOf<kU64> { using T = uint64_t; };
template <> struct DTypeOf<kF64> { using T = double; };

// f(a, b), a the received operand, b the local one; every result is rounded
// to the element type: integers wrap (two's complement), floats round to
// nearest even, 16-bit floats widen to fp32, combine and round once (exact
// for sum by double-rounding innocuity, 24 >= 2p + 2, and for prod because the
// product of two 16-bit values is exact in fp32); max / min keep the received
// operand on ties.
template <class T>
VDEV float widen(T x) {
  if constexpr (std::is_same<T, __half>::value) return __half2float(x);
  else return __bfloat162float(x);
}
template <class T>
VDEV T narrow(float x) {
  if constexpr (std::is_same<T, __half>::value) return __float2half_rn(x);
  else return __float2bfloat16_rn(x);
}
template <class T> struct Is16f {
  static constexpr bool value = std::is_same<T, __half>::value || std::is_same<T, __nv_bfloat16>::value;
};

template <class T, class Op>
struct ElemOp {
  static VDEV T f(T a, T b) {
    if constexpr (Is16f<T>::value) {
      const float x = widen(a), y = widen(b);
      if constexpr (std::is_same<Op, OpSum>::value) return narrow<T>(__fadd_rn(x, y));
      else if constexpr (std::is_same<Op, OpProd>::value) return narrow<T>(__fmul_rn(x, y));
      else if constexpr (std::is_same<Op, OpMax>::value) return (y > x) ? b : a;
      else return (y < x) ? b : a;
    } else if constexpr (std::is_same<T, float>::value) {
      if constexpr (std::is_same<Op, OpSum>::value) return __fadd_rn(a, b);
      else if constexpr (std::is_same<Op, OpProd>::value) return __fmul_rn(a, b);
      else if constexpr (std::is_same<Op, OpMax>::value) return (b > a) ? b : a;
      else return (b < a) ? b : a;
    } else if constexpr (std::is_same<T, double>::value) {
      if constexpr (std::is_same<Op, OpSum>::value) return __dadd_rn(a, b);
      else if constexpr (std::is_same<Op, OpProd>::value) return __dmul_rn(a, b);
      else if constexpr (std::is_same<Op, OpMax>::value) return (b > a) ? b : a;
      else return (b < a) ? b : a;
    } else {   // integers
      using U = typename std::make_unsigned<T>::type;
      if constexpr (std::is_same<Op, OpSum>::value) return (T)(U)((U)a + (U)b);
      else if constexpr (std::is_same<Op, OpProd>::value) return (T)(U)((U)a * (U)b);
      else if constexpr (std::is_same<Op, OpMax>::value) return (b > a) ? b : a;
      else return (b < a) ? b : a;
    }
  }
};
template <class T> struct ElemOp<T, OpNone> {
  static VDEV T f(T a, T) { return a; }
};
template <class T> struct ElemOp<T, OpAvg> {
  static VDEV T f(T a, T b) { return ElemOp<T, OpSum>::f(a, b); }
};

// avg's final step: x / k, integers truncating toward zero, floats rounded
// once to the type (16-bit: an fp32 quotient rounded again, innocuous)
template <class T>
VDEV T divElem(T x, int k) {
  if constexpr (Is16f<T>::value) return narrow<T>(__fdiv_rn(widen(x), (float)k));
  else if constexpr (std::is_same<T, float>::value) return __fdiv_rn(x, (float)k);
  else if constexpr (std::is_same<T, double>::value) return __ddiv_rn(x, (double)k);
  else return (T)(x / (T)k);
}
template <class T, class W>
VDEV W divWord(W w, int k) {
  constexpr int n = sizeof(W) / sizeof(T);
  union U { W w; T e[n]; };
  U u;
  u.w = w;
#pragma unroll
  for (int i = 0; i < n; i++) u.e[i] = divElem<T>(u.e[i], k);
  return u.w;
}

// the sum of two 16-bit lanes per 32-bit word, each lane exactly as
// ElemOp<T, OpSum> computes it (widen to fp32, one fp32 add, round to T with
// RNE), with the two roundings done by one packed conversion
template <class T> VDEV uint32_t sum2(uint32_t a, uint32_t b);
template <> VDEV uint32_t sum2<__nv_bfloat16>(uint32_t a, uint32_t b) {
  const float lo = __fadd_rn(__uint_as_float(a << 16), __uint_as_float(b << 16));
  const float hi = __fadd_rn(__uint_as_float(a & 0xffff0000u), __uint_as_float(b & 0xffff0000u));
  const __nv_bfloat162 r = __float22bfloat162_rn(make_float2(lo, hi));
  return *(const uint32_t*)&r;
}
template <> VDEV uint32_t sum2<__half>(uint32_t a, uint32_t b) {
  const float2 fa = __half22float2(*(const __half2*)&a);
  const float2 fb = __half22float2(*(const __half2*)&b);
  const __half2 r = __float22half2_rn(make_float2(__fadd_rn(fa.x, fb.x), __fadd_rn(fa.y, fb.y)));
  return *(const uint32_t*)&r;
}

// apply f lane-wise on raw words (W = uint4, uint64_t or one element)
template <class T, class Op, class W>
VDEV W applyWord(W a, W b) {
  if constexpr (sizeof(T) == 2 && (std::is_same<Op, OpSum>::value || std::is_same<Op, OpAvg>::value) &&
                sizeof(W) % 4 == 0) {
    constexpr int n = sizeof(W) / 4;
    union U { W w; uint32_t u[n]; };
    U ua, ub, uo;
    ua.w = a;
    ub.w = b;
#pragma unroll
    for (int i = 0; i < n; i++) uo.u[i] = sum2<T>(ua.u[i], ub.u[i]);
    return uo.w;
  } else {
    constexpr int n = sizeof(W) / sizeof(T);
    union U { W w; T e[n]; };
    U ua, ub, uo;
    ua.w = a;
    ub.w = b;
#pragma unroll
    for (int i = 0; i < n; i++) uo.e[i] = ElemOp<T, Op>::f(ua.e[i], ub.e[i]);
    return uo.w;
  }
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
// After ~1024 polls (a few microseconds: a chain's pipeline filling, not a
// step's hand-over) the poller sleeps between polls, so that it stops taking
// issue slots and L2 requests from a CTA moving data on the same SM.
// *seen (if given): the value that satisfied the wait.
VDEV bool waitGeq(const KernArgs& a, const unsigned long long* p, uint64_t v, int rank, int ch,
                  int where, uint64_t* seen = nullptr) {
  uint64_t x = ldAcquire(p);
  if (x >= v) {
    if (seen) *seen = x;
    return true;
  }
  uint64_t t0 = globaltimer();
  unsigned it = 0;
  while (true) {
    x = ldAcquire(p);
    if (x >= v) {
      if (seen) *seen = x;
      return true;
    }
    if (it >= 1024) __nanosleep(128);
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
    if (sizeof(T) == 8) e = *(const uint64_t*)(p + b);
    else if (sizeof(T) == 4) e = *(const uint32_t*)(p + b);
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
    uint64_t e = b < 8 ? v >> (8 * b) : 0;
    if (sizeof(T) == 8) *(uint64_t*)(p + b) = e;
    else if (sizeof(T) == 4) *(uint32_t*)(p + b) = (uint32_t)e;
    else if (sizeof(T) == 2) *(uint16_t*)(p + b) = (uint16_t)e;
    else *(uint8_t*)(p + b) = (uint8_t)e;
  }
}

// ------------------------------------------------------------------ Simple reduce-copy
// d*[i] = fold over the NSRC sources: v = s0[i]; v = f(s1[i], v); v = f(s2[i], v).
// Warp-contiguous 16-byte vectors: a warp owns 32 x UNROLL consecutive packs
// per round (lane l takes packs l, l + 32, ...), so every load instruction is
// one coalesced 512-byte access and all UNROLL x NSRC loads of a round are in
// flight together.  Element-wise tail, and an element-wise path when any
// pointer is not 16-byte aligned.  nbytes < 2^32 (one FIFO slot at most).
// div != 0: the folded value is divided by div before it is stored (avg).
template <class T, class Op, int NSRC>
VDEV void reduceCopy(int tid, int nthr, const char* s0, const char* s1, const char* s2, char* d0,
                     char* d1, char* d2, int nd, uint32_t nbytes, int div = 0) {
  constexpr int UNROLL = (NSRC == 1) ? 8 : (NSRC == 2) ? 4 : 2;
  uintptr_t orall = (uintptr_t)s0 | (uintptr_t)d0;
  if (NSRC > 1) orall |= (uintptr_t)s1;
  if (NSRC > 2) orall |= (uintptr_t)s2;
  if (nd > 1) orall |= (uintptr_t)d1;
  if (nd > 2) orall |= (uintptr_t)d2;
  uint32_t done = 0;
  if ((orall & 15) == 0) {
    const uint32_t npk = nbytes / 16;
    const uint32_t lane = tid & 31, warp = tid >> 5, nwarps = nthr >> 5;
    for (uint32_t base = warp * 32u * UNROLL; base < npk; base += nwarps * 32u * UNROLL) {
      const uint32_t i0 = base + lane;
      const uint4* pa = (const uint4*)s0 + i0;
      const uint4* pb = (const uint4*)s1 + i0;
      const uint4* pc = (const uint4*)s2 + i0;
      uint4 v[UNROLL], w1[UNROLL], w2[UNROLL];
#pragma unroll
      for (int u = 0; u < UNROLL; u++) {
        if (i0 + 32u * u < npk) {
          v[u] = ldCG(pa + 32 * u);
          if (NSRC > 1) w1[u] = ldCG(pb + 32 * u);
          if (NSRC > 2) w2[u] = ldCG(pc + 32 * u);
        }
      }
#pragma unroll
      for (int u = 0; u < UNROLL; u++) {
        if (i0 + 32u * u < npk) {
          if (NSRC > 1) v[u] = applyWord<T, Op>(w1[u], v[u]);
          if (NSRC > 2) v[u] = applyWord<T, Op>(w2[u], v[u]);
          if (div) v[u] = divWord<T>(v[u], div);
          st16((uint4*)d0 + i0 + 32 * u, v[u]);
          if (nd > 1) st16((uint4*)d1 + i0 + 32 * u, v[u]);
          if (nd > 2) st16((uint4*)d2 + i0 + 32 * u, v[u]);
        }
      }
    }
    done = npk * 16;
  }
  const uint32_t ne = (nbytes - done) / (uint32_t)sizeof(T);
  for (uint32_t e = tid; e < ne; e += nthr) {
    const uint32_t off = done + e * (uint32_t)sizeof(T);
    T v = *(const T*)(s0 + off);
    if (NSRC > 1) v = ElemOp<T, Op>::f(*(const T*)(s1 + off), v);
    if (NSRC > 2) v = ElemOp<T, Op>::f(*(const T*)(s2 + off), v);
    if (div) v = divElem<T>(v, div);
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

// warp-collective: v0/v1 already hold one load of this lane's 16 bytes;
// re-load until every valid line of the warp carries `flag`.  false on
// deadline / abort (warp-uniform).
VDEV bool ll128Ready(const KernArgs& a, const char* slot, unsigned long long line, int lane,
                     bool lineValid, uint64_t flag, uint64_t& v0, uint64_t& v1,
                     volatile int* sAbort, int rank, int ch) {
  const int j = lane & 7;
  unsigned it = 0;
  uint64_t t0 = 0;
  while (true) {
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
    if (lineValid) ldVolatile2(slot + 128 * line + 16 * j, v0, v1);
  }
}

// poll an LL line pair whose first load is already in x, y
VDEV bool llReady(const KernArgs& a, const char* slot, unsigned long long p, uint32_t flag,
                  uint64_t& x, uint64_t& y, volatile int* sAbort, int rank, int ch) {
  unsigned it = 0;
  uint64_t t0 = 0;
  while ((uint32_t)(x >> 32) != flag || (uint32_t)(y >> 32) != flag) {
    if (((++it) & 255u) == 0) {
      if (*sAbort) return false;
      if (*a.abortFlag) { reportFailure(a, vAborted, rank, ch, 3); *sAbort = 1; return false; }
      uint64_t now = globaltimer();
      if (t0 == 0) t0 = now;
      else if (now - t0 > a.timeoutNs) { reportFailure(a, vTimeout, rank, ch, 3); *sAbort = 1; return false; }
    }
    ldVolatile2(slot + 16 * p, x, y);
  }
  return true;
}

// ------------------------------------------------------------------ primitives
// One worker's connections, copied once per launch into shared memory, so
// that a step's bookkeeping reads no connection descriptor from global memory
// (the memory clobbers of the flag and counter accesses make the compiler
// re-read such fields at every step, on the step's critical path).  Index i:
// receive connections 0, 1, then send connections 0, 1.
struct ConnCache {
  char* buf[4];                        // the connection's nsteps slots
  unsigned long long* mine[4];         // the counter this worker advances: head (receive), tail (send)
  const unsigned long long* peer[4];   // the counter it waits on: tail (receive), head (send)
  uint64_t credit[2];                  // thread 0: each send connection's head last seen (slots freed)
};

// Shared memory of one CTA's FIFO workers: an abort word per worker group
// (the tree's reduce and broadcast groups stop separately) and a connection
// cache per barrier id (0: the ring worker or tree root; 1, 2: the tree's
// reduce and broadcast groups).
struct WorkerShared {
  int abort[2];
  ConnCache cc[3];
};

// A Prims object is one worker's view of its connections: up to two receive
// connections (all read by a recv* primitive) and up to two send connections
// (all written by a *send primitive).  The seven primitives of Sec. V-B are
// the combinations of (receive?, local input?, send?, user output?).  The
// FIFO positions are kept in scalars so that they stay in registers, and the
// slot each connection's next step uses in one packed word (byte i for
// connection i), advanced with a wrap instead of a modulo.
template <int PROTO, class T, class Op>
struct Prims {
  const KernArgs& a;
  int tid, nthr, barId;
  volatile int* sAbort;
  ConnCache* cc;
  int rank, ch;
  int nrc, nsc;
  uint32_t slots;
  uint64_t rstep0, rstep1, sstep0, sstep1;

  VDEV Prims(const KernArgs& args, int tid_, int nthr_, int barId_, volatile int* sAbort_, ConnCache* cc_,
             int rank_, int ch_, const ConnDev* r0, const ConnDev* r1, const ConnDev* s0, const ConnDev* s1)
      : a(args), tid(tid_), nthr(nthr_), barId(barId_), sAbort(sAbort_), cc(cc_), rank(rank_), ch(ch_) {
    // compact the connection lists: r0/s0 are filled first
    const ConnDev* c[4] = {r0 ? r0 : r1, r0 ? r1 : nullptr, s0 ? s0 : s1, s0 ? s1 : nullptr};
    nrc = (c[0] ? 1 : 0) + (c[1] ? 1 : 0);
    nsc = (c[2] ? 1 : 0) + (c[3] ? 1 : 0);
    // a worker is the only writer of its send conns' tail and its receive
    // conns' head, so their current values are its position in each FIFO
    rstep0 = c[0] ? ldAcquire(c[0]->head) : 0;
    rstep1 = c[1] ? ldAcquire(c[1]->head) : 0;
    sstep0 = c[2] ? ldAcquire(c[2]->tail) : 0;
    sstep1 = c[3] ? ldAcquire(c[3]->tail) : 0;
    const uint64_t ns = (uint64_t)a.nsteps;
    slots = (uint32_t)(rstep0 % ns) | ((uint32_t)(rstep1 % ns) << 8) | ((uint32_t)(sstep0 % ns) << 16) |
            ((uint32_t)(sstep1 % ns) << 24);
    // the other threads of the worker read the cache after the first step's
    // barrier (bar.sync orders shared memory among its threads)
    if (tid == 0) {
#pragma unroll
      for (int i = 0; i < 4; i++) {
        cc->buf[i] = c[i] ? c[i]->buf : nullptr;
        cc->mine[i] = c[i] ? (i < 2 ? c[i]->head : c[i]->tail) : nullptr;
        cc->peer[i] = c[i] ? (i < 2 ? c[i]->tail : c[i]->head) : nullptr;
      }
      cc->credit[0] = cc->credit[1] = 0;
    }
  }

  VDEV void bar() { groupBar(barId, nthr); }
  // connection i's slot for its next step
  VDEV char* slotOf(int i) const {
    return cc->buf[i] + (size_t)((slots >> (8 * i)) & 0xffu) * a.slotBytes;
  }
  // advance the slot indices of connections i and i + 1 by one step
  VDEV void bumpSlots(int i) {
    const uint32_t ns = (uint32_t)a.nsteps;
    uint32_t x = ((slots >> (8 * i)) & 0xffu) + 1, y = ((slots >> (8 * i + 8)) & 0xffu) + 1;
    if (x == ns) x = 0;
    if (y == ns) y = 0;
    slots = (slots & ~(0xffffu << (8 * i))) | (x << (8 * i)) | (y << (8 * i + 8));
  }

  // wait for data (Simple only) and for send credits, then a group barrier
  VDEV bool acquire(bool doRecv, bool doSend) {
    if (tid == 0) {
      bool ok = true;
      if (PROTO == kSimple && doRecv) {
        ok = waitGeq(a, cc->peer[0], rstep0 + 1, rank, ch, 1);
        if (ok && nrc > 1) ok = waitGeq(a, cc->peer[1], rstep1 + 1, rank, ch, 1);
      }
      if (doSend && ok) {
        // a slot is free once the receiver's head has passed it; the head
        // seen last usually covers several steps, so it is read again only
        // when it does not
        const uint64_t ns = (uint64_t)a.nsteps;
        if (sstep0 + 1 > ns && cc->credit[0] < sstep0 + 1 - ns)
          ok = waitGeq(a, cc->peer[2], sstep0 + 1 - ns, rank, ch, 2, &cc->credit[0]);
        if (ok && nsc > 1 && sstep1 + 1 > ns && cc->credit[1] < sstep1 + 1 - ns)
          ok = waitGeq(a, cc->peer[3], sstep1 + 1 - ns, rank, ch, 2, &cc->credit[1]);
      }
      if (!ok) *sAbort = 1;
    }
    bar();
    return *sAbort == 0;
  }

  // publish the step: tail for sends, head for receives.  Simple: every
  // thread's slot writes (and reads) are ordered before thread 0's release
  // store by the block barrier (CTA scope) and carried to the device scope by
  // the release's cumulativity; the receiver acquires the tail and passes its
  // own barrier before any thread reads the slot.  No per-thread fence.
  VDEV bool release(bool doRecv, bool doSend) {
    bar();
    if (*sAbort) return false;
    if (tid == 0) {
      // Simple: one release fence, then every counter of the step with a
      // strong relaxed store (a release pattern for each of them: the slot
      // writes of a send and the slot reads of a receive, ordered before the
      // fence by the barrier above, are seen before the counter).  One fence
      // instead of a release store per counter, whose fences would each wait
      // for the store before it.  LL / LL128 publish data through the lines'
      // flags, so their counters need no fence on the step's path.
      if (PROTO == kSimple) fenceAcqRel();
      if (doSend) {
        stRelaxed(cc->mine[2], sstep0 + 1);
        if (nsc > 1) stRelaxed(cc->mine[3], sstep1 + 1);
      }
      if (doRecv) {
        stRelaxed(cc->mine[0], rstep0 + 1);
        if (nrc > 1) stRelaxed(cc->mine[1], rstep1 + 1);
      }
    }
    if (doSend) { sstep0++; sstep1++; bumpSlots(2); }
    if (doRecv) { rstep0++; rstep1++; bumpSlots(0); }
    return true;
  }

  // one FIFO step of m units (m <= slotUnits)
  VDEV bool step(bool doRecv, bool doLocal, bool doSend, bool doOut, const T* local, T* out,
                 uint32_t m) {
    if (!acquire(doRecv, doSend)) return false;
    const uint32_t nbytes = m * (uint32_t)sizeof(T);
    // avg: the step that both reduces and writes the output completes the
    // value (ring segment owner, tree root, Reduce / ReduceScatter final)
    const int div = (std::is_same<Op, OpAvg>::value && doRecv && doLocal && doOut) ? a.postDiv : 0;
    if (PROTO == kSimple) {
      const char* s0;
      const char* s1 = nullptr;
      const char* s2 = nullptr;
      int ns;
      if (doLocal) {
        s0 = (const char*)local;
        ns = 1;
        if (doRecv) {
          s1 = slotOf(0);
          ns = 2;
          if (nrc > 1) { s2 = slotOf(1); ns = 3; }
        }
      } else {
        s0 = slotOf(0);
        ns = 1;
        if (nrc > 1) { s1 = slotOf(1); ns = 2; }
      }
      char* d0 = nullptr;
      char* d1 = nullptr;
      char* d2 = nullptr;
      int nd = 0;
      if (doOut) { d0 = (char*)out; nd = 1; }
      if (doSend) {
        char* t0 = slotOf(2);
        char* t1 = nsc > 1 ? slotOf(3) : nullptr;
        if (nd == 0) { d0 = t0; d1 = t1; } else { d1 = t0; d2 = t1; }
        nd += nsc;
      }
      if (ns == 1) reduceCopy<T, Op, 1>(tid, nthr, s0, s1, s2, d0, d1, d2, nd, nbytes);
      else if (ns == 2) reduceCopy<T, Op, 2>(tid, nthr, s0, s1, s2, d0, d1, d2, nd, nbytes, div);
      else reduceCopy<T, Op, 3>(tid, nthr, s0, s1, s2, d0, d1, d2, nd, nbytes, div);
    } else if (PROTO == kLL) {
      // each thread owns line pairs p = tid + u * nthr (u < U) per round: all
      // loads of the round are issued before the first flag check
      constexpr int U = 4;
      const uint32_t npairs = (nbytes + 7) / 8;
      const char* rs0 = doRecv ? slotOf(0) : nullptr;
      const char* rs1 = (doRecv && nrc > 1) ? slotOf(1) : nullptr;
      char* ss0 = doSend ? slotOf(2) : nullptr;
      char* ss1 = (doSend && nsc > 1) ? slotOf(3) : nullptr;
      const uint32_t rf0 = (uint32_t)(rstep0 + 1), rf1 = (uint32_t)(rstep1 + 1);
      const uint32_t sf0 = (uint32_t)(sstep0 + 1), sf1 = (uint32_t)(sstep1 + 1);
      bool fail = false;
      for (uint32_t p0 = tid; p0 < npairs && !fail; p0 += (uint32_t)U * nthr) {
        uint64_t v[U], x[U], y[U];
#pragma unroll
        for (int u = 0; u < U; u++) {
          const uint32_t p = p0 + (uint32_t)u * nthr;
          v[u] = 0;
          if (p < npairs) {
            if (doLocal) {
              const int valid = (int)((nbytes - 8 * p) < 8 ? (nbytes - 8 * p) : 8);
              v[u] = loadUser8<T>((const char*)local + 8ull * p, valid);
            }
            if (doRecv) ldVolatile2(rs0 + 16ull * p, x[u], y[u]);
          }
        }
        for (int i = 0; i < (doRecv ? nrc : 0) && !fail; i++) {
          const char* rs = i ? rs1 : rs0;
          const uint32_t rf = i ? rf1 : rf0;
          if (i > 0) {
#pragma unroll
            for (int u = 0; u < U; u++) {
              const uint32_t p = p0 + (uint32_t)u * nthr;
              if (p < npairs) ldVolatile2(rs + 16ull * p, x[u], y[u]);
            }
          }
#pragma unroll
          for (int u = 0; u < U; u++) {
            const uint32_t p = p0 + (uint32_t)u * nthr;
            if (p >= npairs || fail) continue;
            if (!llReady(a, rs, p, rf, x[u], y[u], sAbort, rank, ch)) { fail = true; continue; }
            const uint64_t w = (x[u] & 0xffffffffull) | (y[u] << 32);
            v[u] = (doLocal || i > 0) ? applyWord<T, Op>(w, v[u]) : w;
          }
        }
        if (fail) break;
#pragma unroll
        for (int u = 0; u < U; u++) {
          const uint32_t p = p0 + (uint32_t)u * nthr;
          if (p >= npairs) continue;
          const int valid = (int)((nbytes - 8 * p) < 8 ? (nbytes - 8 * p) : 8);
          if (div) v[u] = divWord<T>(v[u], div);
          if (doOut) storeUser8<T>((char*)out + 8ull * p, v[u], valid);
          if (doSend) {
            llStorePair(ss0, p, v[u], sf0);
            if (nsc > 1) llStorePair(ss1, p, v[u], sf1);
          }
        }
      }
    } else {  // LL128
      // a warp owns line quads q = warp + u * nwarps (u < U) per round; all
      // loads of the round are issued before the first flag check
      constexpr int U = 2;
      const uint32_t nlines = (nbytes + 119) / 120;
      const uint32_t nquads = (nlines + 3) / 4;
      const int warp = tid >> 5, lane = tid & 31, nwarps = nthr >> 5;
      const int j = lane & 7;
      const char* rs0 = doRecv ? slotOf(0) : nullptr;
      const char* rs1 = (doRecv && nrc > 1) ? slotOf(1) : nullptr;
      char* ss0 = doSend ? slotOf(2) : nullptr;
      char* ss1 = (doSend && nsc > 1) ? slotOf(3) : nullptr;
      const uint64_t rf0 = rstep0 + 1, rf1 = rstep1 + 1, sf0 = sstep0 + 1, sf1 = sstep1 + 1;
      uint32_t q0 = warp;
      // Fast path for rounds of UF full line quads when the user pointers
      // are 16-byte aligned.  A half-warp covers a line pair: 240 user bytes,
      // 15 aligned 16-byte chunks, and lane h < 15 of the half loads or
      // stores chunk h in one access.  In the line layout, lanes 0..7 of
      // the first line hold chunks 0..6 and the low half of chunk 7 as they
      // are; lane 8 + j of the second line holds the high half of chunk
      // 7 + j and the low half of chunk 8 + j, which one 64-bit shuffle moves
      // between neighbouring lanes (up on the way in, down on the way out).
      // Same lines, same words, same bits as the element-wise path below.
      if (((((uintptr_t)local) | ((uintptr_t)out)) & 15) == 0) {
        constexpr int UF = 4;
        const uint32_t fullQuads = nbytes / 480;
        const int h = lane & 15;
        const uint32_t hoff = 240u * (uint32_t)(lane >> 4) + 16u * (uint32_t)h;
        for (; q0 + (uint32_t)(UF - 1) * nwarps < fullQuads; q0 += (uint32_t)UF * nwarps) {
          uint64_t v0[UF], v1[UF], w0[UF], w1[UF];
#pragma unroll
          for (int u = 0; u < UF; u++) {
            const uint32_t q = q0 + (uint32_t)u * nwarps;
            const uint32_t line = 4 * q + (lane >> 3);
            v0[u] = 0;
            v1[u] = 0;
            if (doLocal && h < 15) {
              const uint4 c = *(const uint4*)((const char*)local + 480ull * q + hoff);
              v0[u] = ((uint64_t)c.y << 32) | c.x;
              v1[u] = ((uint64_t)c.w << 32) | c.z;
            }
            if (doRecv) ldVolatile2(rs0 + 128ull * line + 16 * j, w0[u], w1[u]);
          }
          if (doLocal) {   // chunk layout -> line layout
#pragma unroll
            for (int u = 0; u < UF; u++) {
              const uint64_t leftHi = __shfl_up_sync(0xffffffffu, v1[u], 1, 16);
              const uint64_t lo = v0[u];
              v0[u] = (h < 8) ? lo : leftHi;
              v1[u] = (h < 7) ? v1[u] : lo;
            }
          }
          bool fail = false;
          for (int i = 0; i < (doRecv ? nrc : 0) && !fail; i++) {
            const char* rs = i ? rs1 : rs0;
            const uint64_t rf = i ? rf1 : rf0;
            if (i > 0) {
#pragma unroll
              for (int u = 0; u < UF; u++) {
                const uint32_t line = 4 * (q0 + (uint32_t)u * nwarps) + (lane >> 3);
                ldVolatile2(rs + 128ull * line + 16 * j, w0[u], w1[u]);
              }
            }
            bool ok = true;
#pragma unroll
            for (int u = 0; u < UF; u++) ok = ok && (j != 7 || w1[u] == rf);
            if (!__all_sync(0xffffffffu, ok)) {
#pragma unroll
              for (int u = 0; u < UF; u++) {
                const uint32_t line = 4 * (q0 + (uint32_t)u * nwarps) + (lane >> 3);
                if (fail) continue;   // warp-uniform
                if (!ll128Ready(a, rs, line, lane, true, rf, w0[u], w1[u], sAbort, rank, ch)) fail = true;
              }
            }
            if (fail) break;
#pragma unroll
            for (int u = 0; u < UF; u++) {
              if (doLocal || i > 0) {
                v0[u] = applyWord<T, Op>(w0[u], v0[u]);
                v1[u] = applyWord<T, Op>(w1[u], v1[u]);
              } else {
                v0[u] = w0[u];
                v1[u] = w1[u];
              }
            }
          }
          if (fail) { q0 = nquads; break; }   // warp-uniform; sAbort records it
#pragma unroll
          for (int u = 0; u < UF; u++) {
            const uint32_t q = q0 + (uint32_t)u * nwarps;
            const uint32_t line = 4 * q + (lane >> 3);
            if (div) {
              v0[u] = divWord<T>(v0[u], div);
              v1[u] = divWord<T>(v1[u], div);
            }
            if (doSend) {
              ll128Store(ss0, line, j, v0[u], v1[u], sf0);
              if (nsc > 1) ll128Store(ss1, line, j, v0[u], v1[u], sf1);
            }
            if (doOut) {   // line layout -> chunk layout
              const uint64_t rightLo = __shfl_down_sync(0xffffffffu, v0[u], 1, 16);
              const uint64_t lo = (h <= 7) ? v0[u] : v1[u];
              const uint64_t hi = (h < 7) ? v1[u] : rightLo;
              if (h < 15)
                st16((char*)out + 480ull * q + hoff,
                     make_uint4((uint32_t)lo, (uint32_t)(lo >> 32), (uint32_t)hi, (uint32_t)(hi >> 32)));
            }
          }
        }
      }
      for (; q0 < nquads; q0 += (uint32_t)U * nwarps) {
        uint64_t v0[U], v1[U], w0[U], w1[U];
        bool lv[U];
        int valid[U];
#pragma unroll
        for (int u = 0; u < U; u++) {
          const uint32_t line = 4 * (q0 + (uint32_t)u * nwarps) + (lane >> 3);
          lv[u] = line < nlines;
          const uint32_t uoff = 120 * line + 16 * j;
          const int cap = (j == 7) ? 8 : 16;
          const int rem = lv[u] ? (int)nbytes - (int)uoff : 0;
          valid[u] = rem <= 0 ? 0 : (rem < cap ? rem : cap);
          v0[u] = 0;
          v1[u] = 0;
          w0[u] = 0;
          w1[u] = 0;
          if (doLocal && valid[u] > 0) {
            v0[u] = loadUser8<T>((const char*)local + uoff, valid[u] < 8 ? valid[u] : 8);
            v1[u] = loadUser8<T>((const char*)local + uoff + 8, valid[u] > 8 ? valid[u] - 8 : 0);
          }
          if (doRecv && lv[u]) ldVolatile2(rs0 + 128ull * line + 16 * j, w0[u], w1[u]);
        }
        bool fail = false;
        for (int i = 0; i < (doRecv ? nrc : 0) && !fail; i++) {
          const char* rs = i ? rs1 : rs0;
          const uint64_t rf = i ? rf1 : rf0;
          if (i > 0) {
#pragma unroll
            for (int u = 0; u < U; u++) {
              const uint32_t line = 4 * (q0 + (uint32_t)u * nwarps) + (lane >> 3);
              if (lv[u]) ldVolatile2(rs + 128ull * line + 16 * j, w0[u], w1[u]);
            }
          }
          // one vote for all lines of the round; flag lanes (j == 7) decide
          bool ok = true;
#pragma unroll
          for (int u = 0; u < U; u++) ok = ok && (!lv[u] || j != 7 || w1[u] == rf);
          if (!__all_sync(0xffffffffu, ok)) {
#pragma unroll
            for (int u = 0; u < U; u++) {
              const uint32_t line = 4 * (q0 + (uint32_t)u * nwarps) + (lane >> 3);
              if (fail) continue;   // warp-uniform
              if (!ll128Ready(a, rs, line, lane, lv[u], rf, w0[u], w1[u], sAbort, rank, ch)) fail = true;
            }
          }
          if (fail) break;
#pragma unroll
          for (int u = 0; u < U; u++) {
            if (doLocal || i > 0) {
              v0[u] = applyWord<T, Op>(w0[u], v0[u]);
              v1[u] = applyWord<T, Op>(w1[u], v1[u]);
            } else {
              v0[u] = w0[u];
              v1[u] = w1[u];
            }
          }
        }
        if (fail) break;   // warp-uniform
#pragma unroll
        for (int u = 0; u < U; u++) {
          const uint32_t line = 4 * (q0 + (uint32_t)u * nwarps) + (lane >> 3);
          const uint32_t uoff = 120 * line + 16 * j;
          if (div) {
            v0[u] = divWord<T>(v0[u], div);
            v1[u] = divWord<T>(v1[u], div);
          }
          if (doOut && valid[u] > 0) {
            storeUser8<T>((char*)out + uoff, v0[u], valid[u] < 8 ? valid[u] : 8);
            storeUser8<T>((char*)out + uoff + 8, v1[u], valid[u] > 8 ? valid[u] - 8 : 0);
          }
          if (doSend && lv[u]) {
            ll128Store(ss0, line, j, v0[u], v1[u], sf0);
            if (nsc > 1) ll128Store(ss1, line, j, v0[u], v1[u], sf1);
          }
        }
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
      if (!step(doRecv, doLocal, doSend, doOut, local + done, out + done, (uint32_t)m)) return false;
      done += m;
    }
    return true;
  }
};

// ------------------------------------------------------------------ schedules
// One primitive invocation: which of (receive, local input, send, user
// output) it uses, and where.  Offsets are in units of the kernel's type.
struct Desc {
  bool recv, local, send, out;
  unsigned long long lo;   // offset into the worker's input buffer
  unsigned long long oo;   // offset into the worker's output buffer
  unsigned long long n;
};

// Worker roles
enum Role : int { kRoleRing = 0, kRoleTreeRoot = 1, kRoleTreeUp = 2, kRoleTreeDown = 3 };

// The step tables of Sec. V-E as an iterator over primitive invocations.
// The ring collectives' block index (r - t - 1) mod k, or (r - t) mod k for
// AllGather, is kept in `blk` and stepped down with a wrap as t advances.
struct Sched {
  int coll, k, r, role, pos;
  bool leaf, inplace;
  unsigned long long count, chunk, end, off, c;
  int t, blk;

  VDEV void init(const KernArgs& a, int r_, int ch, int role_, bool leaf_, int unitBytes) {
    coll = a.coll;
    k = a.nranks;
    r = r_;
    role = role_;
    leaf = leaf_;
    inplace = (a.inplaceMask >> r_) & 1ull;
    count = a.count;
    chunk = a.chunk;
    unsigned long long start, len;
    channelRange(a.count, unitBytes, a.nsub, ch, &start, &len);
    off = start;
    end = start + len;
    t = 0;
    blk = 0;
    c = 0;
    pos = 0;
    if (coll == kBroadcast) pos = modk(r - a.root, k);
    if (coll == kReduce) pos = modk(r - a.root - 1, k);
  }

  VDEV static void set(Desc& d, bool rv, bool lc, bool sd, bool ot) {
    d.recv = rv;
    d.local = lc;
    d.send = sd;
    d.out = ot;
  }

  VDEV bool next(Desc& d, int unitBytes) {
    if (off >= end) return false;
    if (t == 0) blk = (coll == kAllGather) ? r : (r == 0 ? k - 1 : r - 1);
    const int b = blk;   // (r - t - 1) mod k, AllGather (r - t) mod k
    blk = (blk == 0) ? k - 1 : blk - 1;
    if (role == kRoleRing && coll == kAllReduce) {
      // Table "Ring AllReduce": rank r handles segment (r - t - 1) mod k
      if (t == 0) c = ringLoopChunk(off, end, k, chunk, unitBytes);
      const int s = b;
      unsigned long long sa = off + (unsigned long long)s * c;
      if (sa > end) sa = end;
      unsigned long long sb = sa + c;
      if (sb > end) sb = end;
      d.lo = sa;
      d.oo = sa;
      d.n = sb - sa;
      if (t == 0) set(d, false, true, true, false);                 // send
      else if (t <= k - 2) set(d, true, true, true, false);         // recvReduceSend
      else if (t == k - 1) set(d, true, true, true, true);          // recvReduceCopySend
      else if (t <= 2 * k - 3) set(d, true, false, true, true);     // recvCopySend
      else set(d, true, false, false, true);                        // recv
      if (++t > 2 * k - 2) { t = 0; off += (unsigned long long)k * chunk; }
      return true;
    }
    const unsigned long long n = (end - off < chunk) ? end - off : chunk;
    d.n = n;
    if (role == kRoleRing && coll == kReduceScatter) {
      // Table "Ring ReduceScatter": block (r - t - 1) mod k, lands on rank r at t = k-1
      d.lo = (unsigned long long)b * count + off;
      d.oo = off;
      if (t == 0) set(d, false, true, true, false);                 // send
      else if (t <= k - 2) set(d, true, true, true, false);         // recvReduceSend
      else set(d, true, true, false, true);                         // recvReduceCopy
      if (++t > k - 1) { t = 0; off += chunk; }
      return true;
    }
    if (role == kRoleRing && coll == kAllGather) {
      // Table "Ring AllGather": block (r - t) mod k arrives at step t
      d.lo = off;
      d.oo = (unsigned long long)b * count + off;
      if (t == 0) set(d, false, true, true, !inplace);              // send / copySend
      else if (t <= k - 2) set(d, true, false, true, true);         // recvCopySend
      else set(d, true, false, false, true);                        // recv
      if (++t > k - 1) { t = 0; off += chunk; }
      return true;
    }
    d.lo = off;
    d.oo = off;
    off += chunk;
    if (role == kRoleRing && coll == kBroadcast) {
      // Table "Ring Broadcast": root send / copySend, middle recvCopySend, last recv
      if (pos == 0) set(d, false, true, true, !inplace);
      else if (pos < k - 1) set(d, true, false, true, true);
      else set(d, true, false, false, true);
    } else if (role == kRoleRing && coll == kReduce) {
      // Table "Ring Reduce": initiator send, middle recvReduceSend, root recvReduceCopy
      if (pos == 0) set(d, false, true, true, false);
      else if (pos < k - 1) set(d, true, true, true, false);
      else set(d, true, true, false, true);
    } else if (role == kRoleTreeRoot) {
      set(d, true, true, true, true);                                // recvReduceCopySend
    } else if (role == kRoleTreeUp) {
      if (leaf) set(d, false, true, true, false);                    // send
      else set(d, true, true, true, false);                          // recvReduceSend
    } else {
      if (leaf) set(d, true, false, false, true);                    // recv
      else set(d, true, false, true, true);                          // recvCopySend
    }
    return true;
  }
};

// ------------------------------------------------------------------ one worker
// CTA (r, ch) of a collective launch.  Ring collectives: the whole CTA is one
// worker on the ring connections (Sec. V-E tables).  Tree AllReduce (Sec. II-C,
// Table "Tree AllReduce"): sub-channel ch runs tree ch % 2 on its own range;
// the root runs recvReduceCopySend with all its threads, every other rank
// splits its threads into a reduce group (send / recvReduceSend towards the
// root) and a broadcast group (recvCopySend / recv from the root), so the two
// phases stream concurrently.  The data movement has a single call site.
template <int P, class T, class Op>
VDEV void runWorker(const KernArgs& a, int r, int ch, WorkerShared* ws) {
  if (r == a.skipRank) return;   // injected fault: this vrank never takes part
  const int k = a.nranks;
  const ConnDev* r0 = nullptr;
  const ConnDev* r1 = nullptr;
  const ConnDev* s0 = nullptr;
  const ConnDev* s1 = nullptr;
  int tid = threadIdx.x, nthr = blockDim.x, barId = 0, role = kRoleRing;
  bool leaf = false;
  volatile int* ab = ws->abort;
  if (a.algo == kTree) {
    const int t = ch & 1;
    int parent, c0, c1;
    treeLinksM(k, a.treeNode, t, r, &parent, &c0, &c1);
    const ConnDev* up = a.conns + (unsigned long long)ch * k;                   // rank -> parent
    const ConnDev* down = a.conns + a.downOffset + (unsigned long long)ch * k;  // parent -> rank
    leaf = (c0 < 0);
    if (parent < 0) {
      role = kRoleTreeRoot;
      r0 = c0 >= 0 ? &up[c0] : nullptr;
      r1 = c1 >= 0 ? &up[c1] : nullptr;
      s0 = c0 >= 0 ? &down[c0] : nullptr;
      s1 = c1 >= 0 ? &down[c1] : nullptr;
    } else if ((int)threadIdx.x < a.upThreads) {
      role = kRoleTreeUp;
      nthr = a.upThreads;
      barId = 1;
      r0 = c0 >= 0 ? &up[c0] : nullptr;
      r1 = c1 >= 0 ? &up[c1] : nullptr;
      s0 = &up[r];
    } else {
      role = kRoleTreeDown;
      tid = threadIdx.x - a.upThreads;
      nthr = blockDim.x - a.upThreads;
      barId = 2;
      ab = ws->abort + 1;
      r0 = &down[r];
      s0 = c0 >= 0 ? &down[c0] : nullptr;
      s1 = c1 >= 0 ? &down[c1] : nullptr;
    }
  } else {
    const ConnDev* ring = a.conns + (unsigned long long)ch * k;
    bool hasSend = true, hasRecv = true;
    if (a.coll == kBroadcast) {
      const int pos = modk(r - a.root, k);
      hasSend = pos < k - 1;
      hasRecv = pos > 0;
    } else if (a.coll == kReduce) {
      const int pos = modk(r - a.root - 1, k);
      hasSend = pos < k - 1;
      hasRecv = pos > 0;
    }
    s0 = hasSend ? &ring[r] : nullptr;
    r0 = hasRecv ? &ring[modk(r - 1, k)] : nullptr;
  }
  Prims<P, T, Op> pr(a, tid, nthr, barId, ab, &ws->cc[barId], r, ch, r0, r1, s0, s1);
  Sched sc;
  sc.init(a, r, ch, role, leaf, (int)sizeof(T));
  const T* x = (const T*)a.send[r];
  T* y = (T*)a.recv[r];
  Desc d;
  while (sc.next(d, (int)sizeof(T))) {
    if (!pr.run(d.recv, d.local, d.send, d.out, x + d.lo, y + d.oo, d.n)) return;
  }
}

// single-rank communicator: every collective is a copy of the local range
template <class T>
VDEV void localCopy(const KernArgs& a, int ch) {
  unsigned long long start, len;
  channelRange(a.count, sizeof(T), a.nsub, ch, &start, &len);
  if ((a.inplaceMask & 1) || len == 0) return;
  const char* src = (const char*)((const T*)a.send[0] + start);
  char* dst = (char*)((T*)a.recv[0] + start);
  // one slot-sized piece at a time keeps the byte counts within 32 bits
  const unsigned long long piece = 1ull << 30;
  for (unsigned long long o = 0; o < len * sizeof(T); o += piece) {
    const unsigned long long nb = (len * sizeof(T) - o < piece) ? len * sizeof(T) - o : piece;
    reduceCopy<T, OpNone, 1>(threadIdx.x, blockDim.x, src + o, nullptr, nullptr, dst + o, nullptr,
                             nullptr, 1, (uint32_t)nb);
  }
}

}  // namespace vc
