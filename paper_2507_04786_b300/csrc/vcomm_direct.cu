// vcomm_direct.cu -- the direct protocol: collectives with no FIFO.
//
// Sec. IV describes P2P_DIRECT: ranks of one process move data straight
// between source and destination buffers (directSend / directRecv) instead of
// through an intermediate FIFO.  With every vrank in one GPU's memory this
// goes one step further: a thread reads the k input buffers of one 16-byte
// unit itself and folds them in exactly the order the ring schedule would
// (Table "Ring AllReduce": segment s starts at rank s + 1 and ends at rank s;
// ReduceScatter block b likewise from rank b + 1; Reduce from root + 1), so
// the partial sums of the chain never leave registers.  Each input byte is
// read once and each output byte written once: 2kS bytes for a k-vrank
// AllReduce of S bytes per vrank, against 2kS + 4(k-1)S for the Simple ring.
// The segments come from the same partition (channels, loops, chunkCount) as
// the FIFO kernels, so for a given plan the results are the Simple
// protocol's, bit for bit.
//
// No thread waits for another: a plain launch of a grid sized to the data.
#include <cuda_runtime.h>

#include "vcomm_device.cuh"

namespace vc {

namespace {

// the ring segment (fold start = s + 1) of element i of a ring AllReduce,
// and the end (exclusive, in elements) of the run of elements sharing it
VDEV int arSegment(const DirectArgs& a, unsigned long long i, int esz, unsigned long long* runEnd) {
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

template <class T>
struct Unit16 {   // 16-byte unit
  using W = uint4;
  static constexpr int kElems = 16 / sizeof(T);
  static VDEV W load(const char* p) { return __ldcs((const uint4*)p); }
  static VDEV void store(char* p, W v) { __stcs((uint4*)p, v); }
};
template <class T>
struct Unit1 {    // one element (unaligned buffers)
  using W = T;
  static constexpr int kElems = 1;
  static VDEV W load(const char* p) { return *(const T*)p; }
  static VDEV void store(char* p, W v) { *(T*)p = v; }
};

template <class T, class Op, class W>
VDEV W combine(W acc, W x) {
  if constexpr (sizeof(W) == sizeof(T)) return ElemOp<T, Op>::f(acc, x);
  else return applyWord<T, Op>(acc, x);
}

// acc = x_{s+1}; acc = f(acc, x_{s+2}); ... ; acc = f(acc, x_s): the partial
// sum arriving from the predecessor is the first operand, the local input the
// second, as in the FIFO kernels
template <class T, class Op, class U>
VDEV typename U::W foldChain(const DirectArgs& a, int s, unsigned long long off) {
  const int k = a.nranks;
  int r = s + 1 < k ? s + 1 : 0;
  typename U::W acc = U::load((const char*)a.send[r] + off);
  constexpr int B = 8;   // loads issued ahead of their combines
  for (int j = 1; j < k; j += B) {
    typename U::W v[B];
#pragma unroll
    for (int u = 0; u < B; u++) {
      int rr = r + 1 + u;
      if (rr >= k) rr -= k;
      if (j + u < k) v[u] = U::load((const char*)a.send[rr] + off);
    }
#pragma unroll
    for (int u = 0; u < B; u++)
      if (j + u < k) acc = combine<T, Op, typename U::W>(acc, v[u]);
    r += B;
    if (r >= k) r -= k;
  }
  return acc;
}

// the contiguous range of units [*lo, *hi) of this CTA (consecutive threads
// take consecutive units, so every warp access is one coalesced 512 bytes)
VDEV void ctaRange(unsigned long long total, unsigned long long* lo, unsigned long long* hi) {
  unsigned long long per = (total + gridDim.x - 1) / gridDim.x;
  per = (per + blockDim.x - 1) / blockDim.x * blockDim.x;
  *lo = (unsigned long long)blockIdx.x * per;
  *hi = *lo + per < total ? *lo + per : total;
}

// AllReduce, ReduceScatter and Reduce; one unit per loop iteration
template <class T, class Op, class U>
VDEV void directReduce(const DirectArgs& a) {
  const int k = a.nranks;
  constexpr int E = U::kElems;
  const unsigned long long esz = sizeof(T);
  const unsigned long long nunit = a.count / E;                 // full units per block
  const unsigned long long nblk = (a.coll == kReduceScatter) ? (unsigned long long)k : 1ull;
  const unsigned long long total = nunit * nblk;
  unsigned long long lo, hi;
  ctaRange(total, &lo, &hi);
  unsigned long long runEnd = 0;   // AllReduce: the current segment's end (elements)
  int seg = 0;
  for (unsigned long long g = lo + threadIdx.x; g < hi; g += blockDim.x) {
    if (a.coll == kAllReduce) {
      const unsigned long long i = g * E;
      if (i >= runEnd) seg = arSegment(a, i, (int)esz, &runEnd);
      const unsigned long long off = i * esz;
      const typename U::W v = foldChain<T, Op, U>(a, seg, off);
      for (int r = 0; r < k; r++) U::store((char*)a.recv[r] + off, v);
    } else if (a.coll == kReduceScatter) {
      const unsigned long long b = g / nunit, u = g % nunit;
      const typename U::W v = foldChain<T, Op, U>(a, (int)b, (b * a.count + u * E) * esz);
      U::store((char*)a.recv[b] + u * E * esz, v);
    } else {
      const typename U::W v = foldChain<T, Op, U>(a, a.root, g * E * esz);
      U::store((char*)a.recv[a.root] + g * E * esz, v);
    }
  }
  // the element tail of each block (vector units only)
  const unsigned long long tail = a.count - nunit * E;
  if (E > 1 && tail && blockIdx.x == gridDim.x - 1) {
    for (unsigned long long t = threadIdx.x; t < tail * nblk; t += blockDim.x) {
      const unsigned long long b = t / tail, i = nunit * E + t % tail;
      if (a.coll == kAllReduce) {
        unsigned long long re;
        const int s = arSegment(a, i, (int)esz, &re);
        const T v = foldChain<T, Op, Unit1<T>>(a, s, i * esz);
        for (int r = 0; r < k; r++) Unit1<T>::store((char*)a.recv[r] + i * esz, v);
      } else if (a.coll == kReduceScatter) {
        const T v = foldChain<T, Op, Unit1<T>>(a, (int)b, (b * a.count + i) * esz);
        Unit1<T>::store((char*)a.recv[b] + i * esz, v);
      } else {
        const T v = foldChain<T, Op, Unit1<T>>(a, a.root, i * esz);
        Unit1<T>::store((char*)a.recv[a.root] + i * esz, v);
      }
    }
  }
}

template <class T, class Op>
__global__ void __launch_bounds__(256, 2) kDirectReduce(const __grid_constant__ DirectArgs a) {
  if (a.vec) directReduce<T, Op, Unit16<T>>(a);
  else directReduce<T, Op, Unit1<T>>(a);
}

// AllGather (block b of every output = rank b's input) and Broadcast (every
// output = the root's input); count in bytes.  A unit is read once and
// written to every output that is not its own source.
template <class U>
VDEV void directCopy(const DirectArgs& a) {
  const int k = a.nranks;
  constexpr int E = sizeof(typename U::W);
  const unsigned long long nunit = a.count / E;
  const unsigned long long nblk = (a.coll == kAllGather) ? (unsigned long long)k : 1ull;
  const unsigned long long total = nunit * nblk;
  unsigned long long lo, hi;
  ctaRange(total, &lo, &hi);
  for (unsigned long long g = lo + threadIdx.x; g < hi; g += blockDim.x) {
    const unsigned long long b = (a.coll == kAllGather) ? g / nunit : (unsigned long long)a.root;
    const unsigned long long off = (g % nunit) * E;
    const typename U::W v = U::load((const char*)a.send[b] + off);
    const unsigned long long dst = (a.coll == kAllGather) ? b * a.count + off : off;
    for (int r = 0; r < k; r++) {
      if ((unsigned long long)r == b && ((a.inplaceMask >> r) & 1ull)) continue;
      U::store((char*)a.recv[r] + dst, v);
    }
  }
}

__global__ void __launch_bounds__(256) kDirectCopy(const __grid_constant__ DirectArgs a) {
  if (a.vec) {
    directCopy<Unit16<uint8_t>>(a);
    // byte tail of each block
    const unsigned long long nunit = a.count / 16, tail = a.count - nunit * 16;
    const int k = a.nranks;
    const unsigned long long nblk = (a.coll == kAllGather) ? (unsigned long long)k : 1ull;
    if (tail && blockIdx.x == gridDim.x - 1) {
      for (unsigned long long t = threadIdx.x; t < tail * nblk; t += blockDim.x) {
        const unsigned long long b = (a.coll == kAllGather) ? t / tail : (unsigned long long)a.root;
        const unsigned long long off = nunit * 16 + t % tail;
        const uint8_t v = ((const uint8_t*)a.send[b])[off];
        const unsigned long long dst = (a.coll == kAllGather) ? b * a.count + off : off;
        for (int r = 0; r < k; r++) {
          if ((unsigned long long)r == b && ((a.inplaceMask >> r) & 1ull)) continue;
          ((uint8_t*)a.recv[r])[dst] = v;
        }
      }
    }
  } else {
    directCopy<Unit1<uint8_t>>(a);
  }
}

}  // namespace

const void* directKernel(int coll, int dtype, int op) {
  if (coll == kAllGather || coll == kBroadcast) return (const void*)kDirectCopy;
  const bool mx = (op == kMax);
  switch (dtype) {
    case kI32: return mx ? (const void*)kDirectReduce<int32_t, OpMax> : (const void*)kDirectReduce<int32_t, OpSum>;
    case kF32: return mx ? (const void*)kDirectReduce<float, OpMax> : (const void*)kDirectReduce<float, OpSum>;
    case kF16: return mx ? (const void*)kDirectReduce<__half, OpMax> : (const void*)kDirectReduce<__half, OpSum>;
    case kBF16:
      return mx ? (const void*)kDirectReduce<__nv_bfloat16, OpMax> : (const void*)kDirectReduce<__nv_bfloat16, OpSum>;
  }
  return nullptr;
}

}  // namespace vc
