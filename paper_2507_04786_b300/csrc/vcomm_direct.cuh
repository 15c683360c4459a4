// vcomm_direct.cuh -- device code of the direct protocol (no FIFO), shared
// by the per-dtype kernel units (vcomm_direct_inst.cu) and the copy kernels
// (vcomm_direct.cu).  What the protocol computes is described in
// vcomm_direct.cu.
#pragma once
#include "vcomm_device.cuh"

namespace vc {
namespace direct {


// one collective as the direct kernels see it (a single launch or one op of
// a batch): the k send and recv pointers plus DirectArgs' scalars
struct DirectView {
  const void* const* send;
  void* const* recv;
  unsigned long long count, chunk, inplaceMask;
  int coll, nranks, nsub, root;
  int postDiv;   // avg: divide each folded value by this (0: none)
};

// the ring segment (fold start = s + 1) of element i of a ring AllReduce,
// and the end (exclusive, in elements) of the run of elements sharing it
VDEV int arSegment(const DirectView& a, unsigned long long i, int esz, unsigned long long* runEnd) {
  const int k = a.nranks;
  const unsigned long long epp = 16ull / (unsigned long long)esz;
  const unsigned long long npk = a.count / epp;
  const unsigned long long nch = (unsigned long long)a.nsub;
  int ch;
  const unsigned long long q = i / epp;
  if (q >= npk) {
    ch = a.nsub - 1;   // the element tail belongs to the last channel
  } else {
    const unsigned long long base = npk / nch, rem = npk % nch;
    if (q < rem * (base + 1)) ch = (int)(q / (base + 1));
    else ch = (int)(rem + (q - rem * (base + 1)) / base);
  }
  unsigned long long start, len;
  channelRange(a.count, esz, a.nsub, ch, &start, &len);
  const unsigned long long end = start + len;
  const unsigned long long L = (unsigned long long)k * a.chunk;
  const unsigned long long loopOff = start + (i - start) / L * L;
  const unsigned long long c = ringLoopChunk(loopOff, end, k, a.chunk, esz);
  const unsigned long long s = (i - loopOff) / c;
  unsigned long long e = loopOff + (s + 1) * c;
  *runEnd = e < end ? e : end;
  return (int)s;
}

template <class T> struct Unit1;
template <class T>
struct Unit16 {   // 16-byte unit
  using W = uint4;
  using Tail = Unit1<T>;   // the element accesses of the same kernel
  static constexpr int kElems = 16 / sizeof(T);
  static VDEV W load(const char* p) { return __ldcs((const uint4*)p); }
  static VDEV void store(char* p, W v) { __stcs((uint4*)p, v); }
};
template <class T>
struct Unit1 {    // one element (unaligned buffers)
  using W = T;
  using Tail = Unit1<T>;
  static constexpr int kElems = 1;
  static VDEV W load(const char* p) { return *(const T*)p; }
  static VDEV void store(char* p, W v) { *(T*)p = v; }
};

// The same units read through L2 only, for a kernel that outlives the
// requests it serves: a buffer rewritten between two requests must not be
// read from a line that an SM's L1 kept from the earlier one.
template <class T>
struct Unit1L2 {
  using W = T;
  using Tail = Unit1L2<T>;
  static constexpr int kElems = 1;
  static VDEV W load(const char* p) {
    if constexpr (sizeof(T) == 1) {
      unsigned short v;
      asm volatile("ld.global.cg.u8 %0, [%1];" : "=h"(v) : "l"(p));
      const uint8_t b = (uint8_t)v;
      return *(const T*)&b;
    } else if constexpr (sizeof(T) == 2) {
      unsigned short v;
      asm volatile("ld.global.cg.u16 %0, [%1];" : "=h"(v) : "l"(p));
      if constexpr (std::is_same<T, __half>::value) return __ushort_as_half(v);
      else if constexpr (std::is_same<T, __nv_bfloat16>::value) return __ushort_as_bfloat16(v);
      else return (T)v;
    } else if constexpr (sizeof(T) == 4) {
      unsigned v;
      asm volatile("ld.global.cg.u32 %0, [%1];" : "=r"(v) : "l"(p));
      if constexpr (std::is_same<T, float>::value) return __uint_as_float(v);
      else return (T)v;
    } else {
      unsigned long long v;
      asm volatile("ld.global.cg.u64 %0, [%1];" : "=l"(v) : "l"(p));
      if constexpr (std::is_same<T, double>::value) return __longlong_as_double((long long)v);
      else return (T)v;
    }
  }
  static VDEV void store(char* p, W v) { *(T*)p = v; }
};
template <class T>
struct Unit16L2 {
  using W = uint4;
  using Tail = Unit1L2<T>;
  static constexpr int kElems = 16 / sizeof(T);
  static VDEV W load(const char* p) { return ldCG(p); }
  static VDEV void store(char* p, W v) { __stcs((uint4*)p, v); }
};

template <class T, class Op, class W>
VDEV W combine(W acc, W x) {
  if constexpr (sizeof(W) == sizeof(T)) return ElemOp<T, Op>::f(acc, x);
  else return applyWord<T, Op>(acc, x);
}

// acc = x_{s+1}; acc = f(acc, x_{s+2}); ... ; acc = f(acc, x_s): the partial
// sum arriving from the predecessor is the first operand, the local input the
// second, as in the FIFO kernels.  NU units at once (offsets off[u], chain
// starts s[u]): their loads are issued together, B ranks ahead of the combines.
template <class T, class Op, class U, int NU>
VDEV void foldChains(const DirectView& a, const int* s, const unsigned long long* off, int nu,
                     typename U::W* acc) {
  const int k = a.nranks;
  int r[NU];
#pragma unroll
  for (int u = 0; u < NU; u++) {
    r[u] = s[u] + 1 < k ? s[u] + 1 : 0;
    if (u < nu) acc[u] = U::load((const char*)a.send[r[u]] + off[u]);
  }
  constexpr int B = 8;
  for (int j = 1; j < k; j += B) {
    typename U::W v[NU][B];
#pragma unroll
    for (int u = 0; u < NU; u++) {
#pragma unroll
      for (int b = 0; b < B; b++) {
        int rr = r[u] + 1 + b;
        if (rr >= k) rr -= k;
        if (u < nu && j + b < k) v[u][b] = U::load((const char*)a.send[rr] + off[u]);
      }
    }
#pragma unroll
    for (int u = 0; u < NU; u++) {
#pragma unroll
      for (int b = 0; b < B; b++)
        if (u < nu && j + b < k) acc[u] = combine<T, Op, typename U::W>(acc[u], v[u][b]);
      r[u] += B;
      if (r[u] >= k) r[u] -= k;
    }
  }
}

// avg: every value a direct fold produces is complete
template <class T, class U>
VDEV typename U::W divide(typename U::W w, int k) {
  if constexpr (sizeof(typename U::W) == sizeof(T)) return divElem<T>(w, k);
  else return divWord<T>(w, k);
}

template <class T, class Op, class U>
VDEV typename U::W foldChain(const DirectView& a, int s, unsigned long long off) {
  typename U::W acc[1];
  foldChains<T, Op, U, 1>(a, &s, &off, 1, acc);
  return acc[0];
}

// units of a collective: full units per block x blocks
VDEV unsigned long long reduceUnits(const DirectView& a, int E) {
  return (a.count / E) * (a.coll == kReduceScatter ? (unsigned long long)a.nranks : 1ull);
}
VDEV unsigned long long copyUnits(const DirectView& a, int E) {
  return (a.count / E) * (a.coll == kAllGather ? (unsigned long long)a.nranks : 1ull);
}

// The threads that share a range of units: every thread of the CTA (the
// per-call kernels), or the first N (the tile engine's consumer warps; its
// producer warp comes after them).
struct BlockThreads {
  static VDEV unsigned id() { return threadIdx.x; }
  static VDEV unsigned count() { return blockDim.x; }
};
template <unsigned N>
struct FirstThreads {
  static VDEV unsigned id() { return threadIdx.x; }
  static VDEV constexpr unsigned count() { return N; }
};

// AllReduce, ReduceScatter and Reduce over units [lo, hi) of the collective
// (consecutive threads take consecutive units, so every warp access is one
// coalesced 512 bytes), NU units per thread per iteration; `tail`: this CTA
// also does the element tail of each block
template <class T, class Op, class U, int NU, class TS = BlockThreads>
VDEV void directReduce(const DirectView& a, unsigned long long lo, unsigned long long hi, bool tail) {
  const int k = a.nranks;
  constexpr int E = U::kElems;
  const unsigned long long esz = sizeof(T);
  const unsigned long long nunit = a.count / E;                 // full units per block
  unsigned long long runEnd = 0;   // AllReduce: the current segment's end (elements)
  int seg = 0;
  for (unsigned long long g0 = lo + TS::id(); g0 < hi; g0 += (unsigned long long)NU * TS::count()) {
    int s[NU];
    unsigned long long off[NU];
    int nu = 0;
#pragma unroll
    for (int u = 0; u < NU; u++) {
      const unsigned long long g = g0 + (unsigned long long)u * TS::count();
      s[u] = 0;
      off[u] = 0;
      if (g >= hi) continue;
      nu = u + 1;
      if (a.coll == kAllReduce) {
        const unsigned long long i = g * E;
        if (i >= runEnd) seg = arSegment(a, i, (int)esz, &runEnd);
        s[u] = seg;
        off[u] = i * esz;
      } else if (a.coll == kReduceScatter) {
        const unsigned long long b = g / nunit, e = g % nunit;
        s[u] = (int)b;
        off[u] = (b * a.count + e * E) * esz;
      } else {
        s[u] = a.root;
        off[u] = g * E * esz;
      }
    }
    typename U::W v[NU];
    foldChains<T, Op, U, NU>(a, s, off, nu, v);
    if (a.postDiv) {
#pragma unroll
      for (int u = 0; u < NU; u++) v[u] = divide<T, U>(v[u], a.postDiv);
    }
#pragma unroll
    for (int u = 0; u < NU; u++) {
      if (u >= nu) continue;
      if (a.coll == kAllReduce) {
        for (int r = 0; r < k; r++) U::store((char*)a.recv[r] + off[u], v[u]);
      } else if (a.coll == kReduceScatter) {
        const unsigned long long g = g0 + (unsigned long long)u * TS::count();
        U::store((char*)a.recv[s[u]] + (g % nunit) * E * esz, v[u]);
      } else {
        U::store((char*)a.recv[a.root] + off[u], v[u]);
      }
    }
  }
  const unsigned long long nt = a.count - nunit * E;   // element tail of each block
  if (E > 1 && nt && tail) {
    const unsigned long long nblk = (a.coll == kReduceScatter) ? (unsigned long long)k : 1ull;
    for (unsigned long long t = TS::id(); t < nt * nblk; t += TS::count()) {
      const unsigned long long b = t / nt, i = nunit * E + t % nt;
      using U1 = typename U::Tail;
      if (a.coll == kAllReduce) {
        unsigned long long re;
        const int s = arSegment(a, i, (int)esz, &re);
        T v = foldChain<T, Op, U1>(a, s, i * esz);
        if (a.postDiv) v = divElem<T>(v, a.postDiv);
        for (int r = 0; r < k; r++) U1::store((char*)a.recv[r] + i * esz, v);
      } else if (a.coll == kReduceScatter) {
        T v = foldChain<T, Op, U1>(a, (int)b, (b * a.count + i) * esz);
        if (a.postDiv) v = divElem<T>(v, a.postDiv);
        U1::store((char*)a.recv[b] + i * esz, v);
      } else {
        T v = foldChain<T, Op, U1>(a, a.root, i * esz);
        if (a.postDiv) v = divElem<T>(v, a.postDiv);
        U1::store((char*)a.recv[a.root] + i * esz, v);
      }
    }
  }
}

// AllGather (block b of every output = rank b's input) and Broadcast (every
// output = the root's input) over units [lo, hi); count in bytes.  A unit is
// read once and written to every output that is not its own source.
template <class U, class TS = BlockThreads>
VDEV void directCopy(const DirectView& a, unsigned long long lo, unsigned long long hi, bool tail) {
  const int k = a.nranks;
  constexpr int E = sizeof(typename U::W);
  const unsigned long long nunit = a.count / E;
  for (unsigned long long g = lo + TS::id(); g < hi; g += TS::count()) {
    const unsigned long long b = (a.coll == kAllGather) ? g / nunit : (unsigned long long)a.root;
    const unsigned long long off = (g % nunit) * E;
    const typename U::W v = U::load((const char*)a.send[b] + off);
    const unsigned long long dst = (a.coll == kAllGather) ? b * a.count + off : off;
    for (int r = 0; r < k; r++) {
      if ((unsigned long long)r == b && ((a.inplaceMask >> r) & 1ull)) continue;
      U::store((char*)a.recv[r] + dst, v);
    }
  }
  const unsigned long long nt = a.count - nunit * E;   // byte tail of each block
  if (E > 1 && nt && tail) {
    const unsigned long long nblk = (a.coll == kAllGather) ? (unsigned long long)k : 1ull;
    for (unsigned long long t = TS::id(); t < nt * nblk; t += TS::count()) {
      const unsigned long long b = (a.coll == kAllGather) ? t / nt : (unsigned long long)a.root;
      const unsigned long long off = nunit * E + t % nt;
      const uint8_t v = U::Tail::load((const char*)a.send[b] + off);
      const unsigned long long dst = (a.coll == kAllGather) ? b * a.count + off : off;
      for (int r = 0; r < k; r++) {
        if ((unsigned long long)r == b && ((a.inplaceMask >> r) & 1ull)) continue;
        ((uint8_t*)a.recv[r])[dst] = v;
      }
    }
  }
}

// ---- ReduceScatter / AllGather of 16-byte aligned buffers whose blocks are
// not whole 16-byte units (n elements of a block take n x size bytes, not a
// multiple of 16).  Block b then starts (b n size) mod 16 bytes into an
// aligned unit of a send buffer (ReduceScatter) or of the receive buffers
// (AllGather), so the element-wise path would serve them one element per
// access.  Instead every access stays a 16-byte vector: a misaligned
// 16-byte piece is cut out of the two aligned units around it (shiftBytes),
// and the receive buffers are written in aligned units.  Same values, same
// fold order, so the bits are the element-wise path's.

// the 16 bytes that start d bytes (0..15) into the 32 bytes lo:hi
VDEV uint4 shiftBytes(uint4 lo, uint4 hi, unsigned d) {
  const unsigned s = d >> 2, r = (d & 3u) * 8u;
  uint32_t w0, w1, w2, w3, w4;
  if (s == 0) { w0 = lo.x; w1 = lo.y; w2 = lo.z; w3 = lo.w; w4 = hi.x; }
  else if (s == 1) { w0 = lo.y; w1 = lo.z; w2 = lo.w; w3 = hi.x; w4 = hi.y; }
  else if (s == 2) { w0 = lo.z; w1 = lo.w; w2 = hi.x; w3 = hi.y; w4 = hi.z; }
  else { w0 = lo.w; w1 = hi.x; w2 = hi.y; w3 = hi.z; w4 = hi.w; }
  return make_uint4(__funnelshift_r(w0, w1, r), __funnelshift_r(w1, w2, r), __funnelshift_r(w2, w3, r),
                    __funnelshift_r(w3, w4, r));
}

// Memory access policies of the shifted paths: the per-call kernels read
// with plain loads (a thread's two aligned units overlap its neighbours',
// which then come from L1); the resident serving kernel reads through L2 only.
struct PlainMem {
  template <class T> using Elem = Unit1<T>;
  static VDEV uint4 load16(const char* p) { return *(const uint4*)p; }
};
struct L2Mem {
  template <class T> using Elem = Unit1L2<T>;
  static VDEV uint4 load16(const char* p) { return ldCG(p); }
};

// 16 bytes at byte offset x of buffer p of `size` bytes (x + 16 <= size),
// p 16-byte aligned: one or two aligned loads, or byte loads when the second
// aligned unit would reach past the end
template <class M>
VDEV uint4 loadShifted(const char* p, unsigned long long x, unsigned long long size) {
  const unsigned d = (unsigned)(x & 15ull);
  const unsigned long long a0 = x - d;
  if (d == 0) return M::load16(p + a0);
  if (a0 + 32 <= size) return shiftBytes(M::load16(p + a0), M::load16(p + a0 + 16), d);
  union { uint4 v; uint8_t c[16]; } u;
#pragma unroll 1
  for (int i = 0; i < 16; i++) u.c[i] = M::template Elem<uint8_t>::load(p + x + i);
  return u.v;
}

// ReduceScatter units [lo, hi) (16-byte output units of the k blocks, block
// b's full units first), NU units per thread per iteration, 4 ranks at a
// time.  A unit's piece starts d = (b n size) mod 16 bytes into aligned unit
// a0 of every rank's buffer; whether the unit after a0 lies inside the
// buffer is decided once per unit, so the loads of all ranks are issued
// together, without branches, before the first shift (for d = 0 the second
// load repeats the first).  Units whose second aligned unit would pass the
// end of the buffer take loadShifted.  `tail`: this CTA also does each
// block's element tail.
template <class T, class Op, class M, int NU>
VDEV void directReduceShifted(const DirectView& a, unsigned long long lo, unsigned long long hi, bool tail) {
  const int k = a.nranks;
  constexpr int E = 16 / sizeof(T);
  const unsigned long long esz = sizeof(T);
  const unsigned long long nunit = a.count / E;   // full output units per block
  const unsigned long long blockB = a.count * esz, size = blockB * (unsigned long long)k;
  for (unsigned long long g0 = lo + threadIdx.x; g0 < hi; g0 += (unsigned long long)NU * blockDim.x) {
    unsigned long long x[NU], a0[NU], a1[NU], b[NU], e[NU];
    unsigned d[NU];
    int r[NU];
    int nu = 0;
    bool fast = true;
#pragma unroll
    for (int u = 0; u < NU; u++) {
      const unsigned long long g = g0 + (unsigned long long)u * blockDim.x;
      b[u] = 0;
      e[u] = 0;
      x[u] = 0;
      r[u] = 0;
      if (g < hi) {
        nu = u + 1;
        b[u] = g / nunit;
        e[u] = g % nunit;
        x[u] = b[u] * blockB + e[u] * 16ull;
        r[u] = (int)b[u] + 1 < k ? (int)b[u] + 1 : 0;
      }
      d[u] = (unsigned)(x[u] & 15ull);
      a0[u] = x[u] - d[u];
      a1[u] = d[u] ? a0[u] + 16 : a0[u];
      if (g < hi && a0[u] + 32 > size && d[u]) fast = false;
    }
    uint4 acc[NU];
    if (fast) {
      uint4 l0[NU], h0[NU];
#pragma unroll
      for (int u = 0; u < NU; u++) {
        if (u < nu) {
          l0[u] = M::load16((const char*)a.send[r[u]] + a0[u]);
          h0[u] = M::load16((const char*)a.send[r[u]] + a1[u]);
        }
      }
#pragma unroll
      for (int u = 0; u < NU; u++)
        if (u < nu) acc[u] = shiftBytes(l0[u], h0[u], d[u]);
    } else {
#pragma unroll
      for (int u = 0; u < NU; u++)
        if (u < nu) acc[u] = loadShifted<M>((const char*)a.send[r[u]], x[u], size);
    }
    constexpr int B = 4;
    for (int j = 1; j < k; j += B) {
      uint4 vl[NU][B], vh[NU][B];
      if (fast) {
#pragma unroll
        for (int u = 0; u < NU; u++) {
#pragma unroll
          for (int i = 0; i < B; i++) {
            int rr = r[u] + 1 + i;
            if (rr >= k) rr -= k;
            if (u < nu && j + i < k) {
              vl[u][i] = M::load16((const char*)a.send[rr] + a0[u]);
              vh[u][i] = M::load16((const char*)a.send[rr] + a1[u]);
            }
          }
        }
#pragma unroll
        for (int u = 0; u < NU; u++)
#pragma unroll
          for (int i = 0; i < B; i++)
            if (u < nu && j + i < k) vl[u][i] = shiftBytes(vl[u][i], vh[u][i], d[u]);
      } else {
#pragma unroll
        for (int u = 0; u < NU; u++) {
#pragma unroll
          for (int i = 0; i < B; i++) {
            int rr = r[u] + 1 + i;
            if (rr >= k) rr -= k;
            if (u < nu && j + i < k) vl[u][i] = loadShifted<M>((const char*)a.send[rr], x[u], size);
          }
        }
      }
#pragma unroll
      for (int u = 0; u < NU; u++) {
#pragma unroll
        for (int i = 0; i < B; i++)
          if (u < nu && j + i < k) acc[u] = combine<T, Op, uint4>(acc[u], vl[u][i]);
        r[u] += B;
        if (r[u] >= k) r[u] -= k;
      }
    }
#pragma unroll
    for (int u = 0; u < NU; u++) {
      if (u >= nu) continue;
      if (a.postDiv) acc[u] = divide<T, Unit16<T>>(acc[u], a.postDiv);
      *(uint4*)((char*)a.recv[b[u]] + e[u] * 16ull) = acc[u];
    }
  }
  const unsigned long long nt = a.count - nunit * E;   // element tail of each block
  if (nt && tail) {
    using U1 = typename M::template Elem<T>;
    for (unsigned long long t = threadIdx.x; t < nt * (unsigned long long)k; t += blockDim.x) {
      const unsigned long long bl = t / nt, i = nunit * E + t % nt;
      T v = foldChain<T, Op, U1>(a, (int)bl, (bl * a.count + i) * esz);
      if (a.postDiv) v = divElem<T>(v, a.postDiv);
      U1::store((char*)a.recv[bl] + i * esz, v);
    }
  }
}

// AllGather units [lo, hi): the 16-byte units of the k blocks laid end to end
// (count bytes each, not a multiple of 16), each written to every receive
// buffer; `tail`: this CTA also writes the last, partial unit
template <class M, class TS = BlockThreads>
VDEV void directCopyShifted(const DirectView& a, unsigned long long lo, unsigned long long hi, bool tail) {
  using UB = typename M::template Elem<uint8_t>;
  const int k = a.nranks;
  const unsigned long long B = a.count, total = B * (unsigned long long)k;
  for (unsigned long long u = lo + TS::id(); u < hi; u += TS::count()) {
    const unsigned long long x = u * 16ull, b = x / B, o = x - b * B;
    uint4 v;
    if (o + 16 <= B) {
      v = loadShifted<M>((const char*)a.send[b], o, B);
    } else {   // the unit straddles two blocks: byte by byte
      union { uint4 w; uint8_t c[16]; } t;
#pragma unroll 1
      for (int i = 0; i < 16; i++) {
        const unsigned long long y = x + i, bb = y / B;
        t.c[i] = UB::load((const char*)a.send[bb] + (y - bb * B));
      }
      v = t.w;
    }
    for (int r = 0; r < k; r++) *(uint4*)((char*)a.recv[r] + x) = v;
  }
  const unsigned long long full = total / 16ull;
  if (tail && full * 16ull < total) {
    for (unsigned long long y = full * 16ull + TS::id(); y < total; y += TS::count()) {
      const unsigned long long bb = y / B;
      const uint8_t c = UB::load((const char*)a.send[bb] + (y - bb * B));
      for (int r = 0; r < k; r++) ((uint8_t*)a.recv[r])[y] = c;
    }
  }
}

// units of the shifted paths
VDEV unsigned long long shiftedUnits(const DirectView& a, int esz) {
  if (a.coll == kAllGather) return a.count * (unsigned long long)a.nranks / 16ull;
  return (a.count / (16ull / (unsigned long long)esz)) * (unsigned long long)a.nranks;
}

// this CTA's contiguous share [*lo, *hi) of `total` units, in whole blocks
VDEV void ctaRange(unsigned long long total, unsigned long long* lo, unsigned long long* hi) {
  unsigned long long per = (total + gridDim.x - 1) / gridDim.x;
  per = (per + blockDim.x - 1) / blockDim.x * blockDim.x;
  *lo = (unsigned long long)blockIdx.x * per;
  if (*lo > total) *lo = total;
  *hi = *lo + per < total ? *lo + per : total;
}

VDEV DirectView viewOf(const DirectArgs& a) {
  return DirectView{a.send, a.recv, a.count, a.chunk, a.inplaceMask, a.coll, a.nranks, a.nsub, a.root,
                    a.postDiv};
}

// Launch shape (measured on 8 x 256 MiB): 4-byte types keep 4 units x 8
// loads in flight per thread in 256-thread CTAs (1- and 8-byte types too);
// 16-bit floats, whose widened arithmetic needs more issue slots, 2 units in
// 512-thread CTAs.
template <class T> struct DirectShape {
  static constexpr int kUnits = sizeof(T) == 2 ? 2 : 4;
  static constexpr int kThreads = sizeof(T) == 2 ? 512 : 256;
};
inline int directThreadsFor(int esz) { return esz == 2 ? 512 : 256; }

// ---- many direct collectives of one element type and op in one launch
// (group calls; the host launches one such kernel per (dtype, op) present,
// and one for the copies).  The ops' units are laid end to end (op i owns
// [unitStart[i], unitStart[i + 1])); each CTA takes a contiguous share of
// that space and runs every op it overlaps on the overlapping units.
// Nothing waits, so the ops need no ordering.
VDEV DirectView viewOfOp(const DirectBatchArgs* b, int i) {
  const DirectOpDesc& o = b->ops[i];
  return DirectView{(const void* const*)&b->ptrs[o.ptrBase], (void* const*)&b->ptrs[o.ptrBase + o.nranks],
                    o.count, o.chunk, o.inplaceMask, o.coll, o.nranks, o.nsub, o.root, o.postDiv};
}

// the op-local units [lo, hi) of op i that fall in this CTA's share
// [glo, ghi), and whether this CTA holds the op's last unit (its tails)
VDEV void opShare(const DirectBatchArgs* b, int i, unsigned long long glo, unsigned long long ghi,
                  unsigned long long* lo, unsigned long long* hi, bool* tail) {
  const unsigned long long s = b->unitStart[i], e = b->unitStart[i + 1];
  unsigned long long h = (ghi < e ? ghi : e) - s;
  if (h > b->ops[i].units) h = b->ops[i].units;   // the range may hold one unit more than the op
  unsigned long long l = (glo > s ? glo : s) - s;
  *lo = l < h ? l : h;
  *hi = h;
  *tail = ghi >= e;
}


// ---- the reducing collectives staged through shared memory.
//
// Same arithmetic as directReduce (each 16-byte unit's chain folded in its
// ring order), but the data moves by bulk asynchronous copies:
// one thread loads tile i of every rank's input into shared memory (k copies
// that complete one mbarrier), S = a.stages tiles ahead of the fold, and
// stores the folded tile to every rank's output with k bulk stores, so the
// loads in flight never drain while the CTA folds.  Each CTA takes tiles
// blockIdx.x, blockIdx.x + gridDim.x, ...  Shared memory: in[S][k][tile],
// out[2][tile] (the folded tile, double buffered so the stores of one tile
// overlap the fold of the next), then S mbarriers.
constexpr int kMaxStages = 3;

VDEV unsigned smemU32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

VDEV void mbarInit(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smemU32(bar)), "r"(count) : "memory");
}
// the initialised barriers become visible to the bulk-copy (async) proxy
VDEV void fenceBarrierInit() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
// arrive once, expecting `bytes` of bulk copies to complete this phase
VDEV void mbarExpect(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smemU32(bar)), "r"(bytes)
               : "memory");
}
VDEV bool mbarTryWait(uint64_t* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smemU32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// global -> shared, `bytes` (a multiple of 16, both addresses 16-byte aligned)
VDEV void bulkLoad(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smemU32(dst)),
      "l"(src), "r"(bytes), "r"(smemU32(bar))
      : "memory");
}
// shared -> global, same rules
VDEV void bulkStore(void* dst, const void* src, unsigned bytes) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst), "r"(smemU32(src)),
               "r"(bytes)
               : "memory");
}
VDEV void bulkCommit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// every group but the newest has finished reading its shared memory
VDEV void bulkWaitRead1() { asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory"); }
// every group has completed
VDEV void bulkWaitAll() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
// this thread's generic-proxy writes to shared memory become visible to bulk copies
VDEV void fenceProxyAsync() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

VDEV void stagedFailure(const DirectArgs& a, int where) {
  if (atomicCAS(a.errClaim, 0, (int)vTimeout) == 0) {
    volatile ErrWord* e = a.err;
    e->rank = -1;
    e->channel = (int)blockIdx.x;
    e->where = where;
    __threadfence_system();
    e->code = (int)vTimeout;
    __threadfence_system();
  }
}

// wait for phase `parity` of *bar, at most timeoutNs
VDEV bool stageWait(uint64_t* bar, unsigned parity, unsigned long long timeoutNs) {
  if (mbarTryWait(bar, parity)) return true;
  const uint64_t t0 = globaltimer();
  while (true) {
    if (mbarTryWait(bar, parity)) return true;
    if (globaltimer() - t0 > timeoutNs) return false;
  }
}

// AllReduce, ReduceScatter and Reduce staged through shared memory.  A
// tile is a range of one block: the whole buffer (AllReduce, Reduce) or
// block b of the k ReduceScatter blocks (b's chain starts at rank b + 1 and
// ends in recvbuf b); AllReduce units take their segment's chain and go to
// every output, Reduce units the chain ending at the root.
template <class T, class Op>
VDEV void directReduceStaged(const DirectArgs& a) {
  extern __shared__ __align__(128) unsigned char smem[];
  const DirectView v = viewOf(a);
  const int k = a.nranks;
  constexpr int E = Unit16<T>::kElems;
  constexpr unsigned long long esz = sizeof(T);
  const unsigned long long fullBytes = (a.count / E) * 16ull;   // the 16-byte units of a block
  const unsigned tile = (unsigned)a.tileBytes;
  const int S = a.stages;
  const bool rs = a.coll == kReduceScatter;
  const unsigned long long blockStride = rs ? a.count * esz : 0ull;   // between send blocks
  const unsigned long long perBlock = (fullBytes + tile - 1) / tile;
  const unsigned long long ntiles = (rs ? (unsigned long long)k : 1ull) * perBlock;
  unsigned char* in = smem;
  unsigned char* out = smem + (size_t)S * k * tile;
  uint64_t* bar = (uint64_t*)(out + 2 * (size_t)tile);

  // self-check of what the bulk copies need: 16-byte aligned buffers, tiles
  // and shared memory, and one phase's bytes within an mbarrier's count
  bool bad = (smemU32(smem) & 15u) || (tile & 127u) || tile == 0 || S < 2 || S > kMaxStages ||
             (unsigned long long)k * tile >= (1ull << 20) || (blockStride & 15u) ||
             !(a.coll == kAllReduce || rs || a.coll == kReduce);
  for (int r = 0; r < k; r++)
    if (((uintptr_t)v.send[r] | (uintptr_t)v.recv[r]) & 15u) bad = true;
  if (bad) {
    if (threadIdx.x == 0) stagedFailure(a, 5);
    return;
  }
  if (threadIdx.x == 0) {
    for (int s = 0; s < S; s++) mbarInit(&bar[s], 1);
    fenceBarrierInit();
  }
  __syncthreads();

  const unsigned long long G = gridDim.x;
  const unsigned long long mine = blockIdx.x < ntiles ? (ntiles - 1 - blockIdx.x) / G + 1 : 0;
  // my i-th tile: global tile blockIdx.x + i * G = block b, offset off in it
  auto tileAt = [&](unsigned long long i, int* b, unsigned long long* off, unsigned* len) {
    const unsigned long long t = blockIdx.x + i * G;
    *b = (int)(t / perBlock);
    *off = (t % perBlock) * (unsigned long long)tile;
    *len = (unsigned)(fullBytes - *off < tile ? fullBytes - *off : tile);
  };
  auto issue = [&](unsigned long long i) {   // thread 0: the k input tiles of my i-th tile
    const int st = (int)(i % S);
    int b;
    unsigned long long off;
    unsigned len;
    tileAt(i, &b, &off, &len);
    const unsigned long long src = (unsigned long long)b * blockStride + off;
    mbarExpect(&bar[st], len * (unsigned)k);
    for (int r = 0; r < k; r++)
      bulkLoad(in + ((size_t)st * k + r) * tile, (const char*)v.send[r] + src, len, &bar[st]);
  };
  if (threadIdx.x == 0)
    for (unsigned long long i = 0; i < mine && i < (unsigned long long)S; i++) issue(i);

  unsigned long long runEnd = 0;   // the current segment's end (elements); offsets only grow
  int seg = 0;
  unsigned long long i = 0;
  bool failed = false;
  for (; i < mine; i++) {
    const int st = (int)(i % S);
    const bool ok = stageWait(&bar[st], (unsigned)((i / S) & 1ull), a.timeoutNs);
    if (__syncthreads_or(!ok)) {
      failed = true;
      break;
    }
    const int ob = (int)(i & 1ull);
    if (threadIdx.x == 0) bulkWaitRead1();   // the stores of tile i - 2 no longer read out[ob]
    __syncthreads();
    int b;
    unsigned long long off;
    unsigned len;
    tileAt(i, &b, &off, &len);
    const unsigned char* src = in + (size_t)st * k * tile;
    unsigned char* o = out + (size_t)ob * tile;
    for (unsigned u = threadIdx.x * 16u; u < len; u += blockDim.x * 16u) {
      if (a.coll == kAllReduce) {
        const unsigned long long e0 = (off + u) / esz;
        if (e0 >= runEnd) seg = arSegment(v, e0, (int)esz, &runEnd);
      } else {
        seg = rs ? b : a.root;
      }
      int r = seg + 1 < k ? seg + 1 : 0;
      uint4 acc = *(const uint4*)(src + (size_t)r * tile + u);
      for (int j = 1; j < k; j++) {
        if (++r == k) r = 0;
        acc = combine<T, Op, uint4>(acc, *(const uint4*)(src + (size_t)r * tile + u));
      }
      if (a.postDiv) acc = divide<T, Unit16<T>>(acc, a.postDiv);
      *(uint4*)(o + u) = acc;
    }
    fenceProxyAsync();
    __syncthreads();   // out[ob] written; in[st] read by every thread
    if (threadIdx.x == 0) {
      if (a.coll == kAllReduce) {
        for (int r = 0; r < k; r++) bulkStore((char*)v.recv[r] + off, o, len);
      } else {
        bulkStore((char*)v.recv[rs ? b : a.root] + off, o, len);
      }
      bulkCommit();
      if (i + S < mine) issue(i + S);
    }
  }
  if (threadIdx.x == 0) {
    bulkWaitAll();
    if (failed) {
      stagedFailure(a, 4);
      // loads still in flight (tiles i .. i + S - 1) must land before the
      // CTA's shared memory is released
      for (unsigned long long j = i; j < mine && j < i + S; j++)
        (void)stageWait(&bar[j % S], (unsigned)((j / S) & 1ull), a.timeoutNs);
    }
  }
  if (failed) return;
  // the element tail after the last full unit (ReduceScatter blocks of
  // whole units have none)
  if (blockIdx.x == gridDim.x - 1 && !rs) {
    const unsigned long long nunit = a.count / E;
    directReduce<T, Op, Unit16<T>, 1>(v, nunit, nunit, true);
  }
}


// ---- copies staged through shared memory (AllGather, Broadcast, point to
// point).  A copy needs no arithmetic, so one thread per CTA moves the data
// with bulk copies alone: tile i of its share goes global -> shared (one
// mbarrier per stage) and shared -> every destination (bulk stores); the
// load of tile i + S - 1 is issued as soon as the stores of tile i - 1 have
// read their stage, so S - 1 tiles of loads stay in flight.
constexpr int kMaxCopyStages = 4;

VDEV void copyFailure(const CopyArgs& a, int where) {
  if (atomicCAS(a.errClaim, 0, (int)vTimeout) == 0) {
    volatile ErrWord* e = a.err;
    e->rank = -1;
    e->channel = (int)blockIdx.x;
    e->where = where;
    __threadfence_system();
    e->code = (int)vTimeout;
    __threadfence_system();
  }
}

// the task holding global tile t, searching up from task `from` (<= it)
VDEV int copyTaskOf(const CopyArgs& a, unsigned long long t, int from) {
  while (from + 1 < a.ntasks && a.tasks[from + 1].tileStart <= t) from++;
  return from;
}

VDEV void copyStaged(const CopyArgs& a) {
  if (threadIdx.x != 0) return;   // one thread drives the bulk copies
  extern __shared__ __align__(128) unsigned char smem[];
  const unsigned tile = (unsigned)a.tile;
  const int S = a.stages;
  uint64_t* bar = (uint64_t*)(smem + (size_t)S * tile);

  // self-check of what the bulk copies need: 16-byte aligned sources,
  // destinations, offsets and sizes, tiles within an mbarrier's count
  bool bad = (smemU32(smem) & 15u) || (tile & 127u) || tile == 0 || tile >= (1u << 20) || S < 2 ||
             S > kMaxCopyStages || a.ntasks < 1 || a.ntasks > kMaxCopyTasks;
  for (int t = 0; !bad && t < a.ntasks; t++) {
    const CopyTask& c = a.tasks[t];
    if (((uintptr_t)c.src | c.bytes | c.dstOff) & 15u) bad = true;
    if (c.dstBase < 0 || c.ndst < 0 || c.dstBase + c.ndst > kMaxCopyTasks) bad = true;
    for (int d = 0; !bad && d < c.ndst; d++)
      if ((uintptr_t)a.dsts[c.dstBase + d] & 15u) bad = true;
  }
  if (bad) {
    copyFailure(a, 5);
    return;
  }
  for (int s = 0; s < S; s++) mbarInit(&bar[s], 1);
  fenceBarrierInit();

  const unsigned long long G = gridDim.x;
  const unsigned long long mine = blockIdx.x < a.ntiles ? (a.ntiles - 1 - blockIdx.x) / G + 1 : 0;
  // my i-th tile is global tile blockIdx.x + i * G; loads and stores each
  // walk their tiles in increasing order, so each keeps its own task hint
  int loadTask = 0, storeTask = 0;
  auto issue = [&](unsigned long long i) {
    const unsigned long long t = blockIdx.x + i * G;
    loadTask = copyTaskOf(a, t, loadTask);
    const CopyTask& c = a.tasks[loadTask];
    const unsigned long long off = (t - c.tileStart) * (unsigned long long)tile;
    const unsigned len = (unsigned)(c.bytes - off < tile ? c.bytes - off : tile);
    const int st = (int)(i % S);
    mbarExpect(&bar[st], len);
    bulkLoad(smem + (size_t)st * tile, (const char*)c.src + off, len, &bar[st]);
  };
  unsigned long long issued = 0;
  for (; issued < mine && issued + 1 < (unsigned long long)S; issued++) issue(issued);

  unsigned long long i = 0;
  bool failed = false;
  for (; i < mine; i++) {
    const int st = (int)(i % S);
    if (!stageWait(&bar[st], (unsigned)((i / S) & 1ull), a.timeoutNs)) {
      failed = true;
      break;
    }
    const unsigned long long t = blockIdx.x + i * G;
    storeTask = copyTaskOf(a, t, storeTask);
    const CopyTask& c = a.tasks[storeTask];
    const unsigned long long off = (t - c.tileStart) * (unsigned long long)tile;
    const unsigned len = (unsigned)(c.bytes - off < tile ? c.bytes - off : tile);
    for (int d = 0; d < c.ndst; d++)
      if (!((c.skipMask >> d) & 1ull))
        bulkStore((char*)a.dsts[c.dstBase + d] + c.dstOff + off, smem + (size_t)st * tile, len);
    bulkCommit();
    bulkWaitRead1();   // the stores of tile i - 1 have read their stage
    if (issued < mine) issue(issued++);
  }
  bulkWaitAll();
  if (failed) {
    copyFailure(a, 4);
    // loads still in flight (tiles i .. issued - 1) must land before the
    // CTA's shared memory is released
    for (unsigned long long j = i; j < issued; j++)
      (void)stageWait(&bar[j % S], (unsigned)((j / S) & 1ull), a.timeoutNs);
  }
}

}  // namespace direct
}  // namespace vc
