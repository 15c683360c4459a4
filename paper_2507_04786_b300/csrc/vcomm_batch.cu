// vcomm_batch.cu -- the batched launch: many collectives, one persistent kernel.
//
// Group calls (Sec. II-A-4) defer a sequence of collectives so that they run
// as ONE launch.  The grid is a set of gangs; each gang is nranks x cpg CTAs
// and runs its ops one after another on its own channels, so ops of different
// gangs overlap on the device while ops of one gang pipeline through the same
// FIFOs.  CTA (r, ch) of a gang copies each op's description into shared
// memory (the paper's metadata-loading warp, Sec. V-D) and runs the op's
// (protocol, dtype, op) worker; CTAs whose channel the op does not use skip it.
#include <cuda_runtime.h>

#include "vcomm_device.cuh"
#include "vcomm_direct.cuh"
#include "vcomm_kernels.h"

namespace vc {

#define VC_DTYPES_OF(X, P) X(P, 0) X(P, 1) X(P, 2) X(P, 3) X(P, 4) X(P, 5) X(P, 6) X(P, 7) X(P, 8) X(P, 9)
#define VC_DECL(P, D) __device__ void batchWorker_##P##_##D(const KernArgs&, int, int, WorkerShared*);
VC_DTYPES_OF(VC_DECL, 0) VC_DTYPES_OF(VC_DECL, 1) VC_DTYPES_OF(VC_DECL, 2)
#undef VC_DECL

template <int P>
__device__ __noinline__ void batchCopyWorker(const KernArgs& a, int r, int ch, WorkerShared* ws) {
  if (a.coll == kCopy) localCopy<uint8_t>(a, ch);
  else runWorker<P, uint8_t, OpNone>(a, r, ch, ws);
}

__device__ __forceinline__ void dispatchOp(const KernArgs& a, int proto, int dtype, bool bytes,
                                           int r, int ch, WorkerShared* ws) {
  if (bytes) {
    if (proto == kSimple) batchCopyWorker<kSimple>(a, r, ch, ws);
    else if (proto == kLL) batchCopyWorker<kLL>(a, r, ch, ws);
    else batchCopyWorker<kLL128>(a, r, ch, ws);
    return;
  }
#define VC_CASE(P, D) if (proto == P && dtype == D) { batchWorker_##P##_##D(a, r, ch, ws); return; }
  VC_DTYPES_OF(VC_CASE, 0) VC_DTYPES_OF(VC_CASE, 1) VC_DTYPES_OF(VC_CASE, 2)
#undef VC_CASE
}

__global__ void __launch_bounds__(512, 1) kBatch(const __grid_constant__ BatchArgs b) {
  __shared__ KernArgs sa;
  __shared__ WorkerShared ws;
  volatile int* sAbort = ws.abort;
  const int k = b.nranks;
  const int per = k * b.cpg;
  const int gang = blockIdx.x / per;
  const int local = blockIdx.x % per;
  const int ch = local / k;
  const int r = local % k;
  if (threadIdx.x < 2) sAbort[threadIdx.x] = 0;
  for (int i = b.gangStart[gang]; i < b.gangStart[gang + 1]; i++) {
    const BatchOpDesc& o = b.ops[b.order[i]];
    if (ch >= o.nsub) continue;          // the op does not use this channel
    __syncthreads();                     // every thread is done with the previous op's sa
    if (threadIdx.x < k) {
      sa.send[threadIdx.x] = b.ptrs[o.ptrBase + threadIdx.x];
      sa.recv[threadIdx.x] = const_cast<void*>(b.ptrs[o.ptrBase + k + threadIdx.x]);
    }
    if (threadIdx.x == 0) {
      sa.count = o.count;
      sa.chunk = o.chunk;
      sa.slotBytes = o.slotBytes;
      sa.slotUnits = o.slotUnits;
      sa.timeoutNs = b.timeoutNs;
      sa.conns = o.conns ? const_cast<ConnDev*>(o.conns) + (unsigned long long)gang * b.cpg * k : nullptr;
      sa.errClaim = b.errClaim;
      sa.err = b.err;
      sa.abortFlag = b.abortFlag;
      sa.inplaceMask = o.inplaceMask;
      sa.downOffset = o.downOffset;
      sa.coll = o.coll;
      sa.algo = o.algo;
      sa.redop = o.redop;
      sa.nranks = k;
      sa.nsub = o.nsub;
      sa.root = o.root;
      sa.nsteps = b.nsteps;
      sa.upThreads = (blockDim.x / 2) / 32 * 32;
      sa.skipRank = -1;
      sa.postDiv = o.postDiv;
      sa.treeNode = b.treeNode;
    }
    __syncthreads();
    const bool bytes = (o.coll == kAllGather || o.coll == kBroadcast ||
                        (o.coll == kCopy && o.dtype < 0));
    dispatchOp(sa, o.proto, o.dtype, bytes, r, ch, &ws);
    __syncthreads();
    if (sAbort[0] || sAbort[1]) return;  // a wait failed: the error word says where
  }
}

// ---- serving kernel ---------------------------------------------------------
// Every gang loops: its leader CTA waits for the host to post request `seq` in
// the gang's mailbox, copies it to device memory and publishes it; the gang's
// CTAs that the request uses run it (same workers as the batch kernel); all
// CTAs of the gang meet at a barrier, after which the leader reports
// completion to the host.  Waits are bounded: an idle gang stops after
// idleTimeoutNs, a failed one stops and flags its mailbox.
__device__ __forceinline__ uint64_t ldVol64(const volatile unsigned long long* p) { return *p; }

// A request with the direct protocol (no FIFO) spreads its units over all of
// the gang's CTAs: CTA `local` of `nctas` takes a contiguous share.  One body
// per (dtype, op), not inlined, so that each keeps its own registers.
__device__ void shareRange(unsigned long long total, unsigned long long local, unsigned long long nctas,
                           unsigned long long* lo, unsigned long long* hi) {
  unsigned long long per = (total + nctas - 1) / nctas;
  per = (per + blockDim.x - 1) / blockDim.x * blockDim.x;
  *lo = local * per < total ? local * per : total;
  *hi = *lo + per < total ? *lo + per : total;
}

template <class T, class Op>
__device__ __noinline__ void serveDirect(const ServeReq* q, unsigned long long local, unsigned long long nctas) {
  using namespace direct;
  const DirectView v{(const void* const*)q->send, (void* const*)q->recv, q->count, q->chunk, q->inplaceMask,
                     q->coll, q->nranks, q->nsub, q->root, 0};
  unsigned long long lo, hi;
  if (q->coll == kAllGather || q->coll == kBroadcast) {
    if (q->vec) {
      shareRange(copyUnits(v, 16), local, nctas, &lo, &hi);
      directCopy<Unit16<uint8_t>>(v, lo, hi, local + 1 == nctas);
    } else {
      shareRange(copyUnits(v, 1), local, nctas, &lo, &hi);
      directCopy<Unit1<uint8_t>>(v, lo, hi, local + 1 == nctas);
    }
  } else if (q->vec) {
    shareRange(reduceUnits(v, Unit16<T>::kElems), local, nctas, &lo, &hi);
    directReduce<T, Op, Unit16<T>, 1>(v, lo, hi, local + 1 == nctas);
  } else {
    shareRange(reduceUnits(v, 1), local, nctas, &lo, &hi);
    directReduce<T, Op, Unit1<T>, 1>(v, lo, hi, local + 1 == nctas);
  }
}

__device__ void dispatchDirect(const ServeReq* q, unsigned long long local, unsigned long long nctas) {
  const bool mx = q->redop == kMax;
  if (q->coll == kAllGather || q->coll == kBroadcast) serveDirect<uint8_t, OpNone>(q, local, nctas);
  else if (q->dtype == kI32) mx ? serveDirect<int32_t, OpMax>(q, local, nctas) : serveDirect<int32_t, OpSum>(q, local, nctas);
  else if (q->dtype == kF32) mx ? serveDirect<float, OpMax>(q, local, nctas) : serveDirect<float, OpSum>(q, local, nctas);
  else if (q->dtype == kF16) mx ? serveDirect<__half, OpMax>(q, local, nctas) : serveDirect<__half, OpSum>(q, local, nctas);
  else mx ? serveDirect<__nv_bfloat16, OpMax>(q, local, nctas) : serveDirect<__nv_bfloat16, OpSum>(q, local, nctas);
}

__global__ void __launch_bounds__(512, 1) kServe(const __grid_constant__ ServeArgs s) {
  __shared__ KernArgs sa;
  __shared__ WorkerShared ws;
  volatile int* sAbort = ws.abort;
  __shared__ int sStop;
  __shared__ int sUse;
  __shared__ int sCh;
  __shared__ int sR;
  int g = 0;
  while (g + 1 < s.ngangs && (int)blockIdx.x >= s.gangCta[g + 1]) g++;
  const int local = blockIdx.x - s.gangCta[g];
  int ch = 0, r = 0;   // this CTA's (channel, vrank) in the current request
  const unsigned long long nctas = (unsigned long long)(s.gangCta[g + 1] - s.gangCta[g]);
  const bool leader = (local == 0);
  ServeGang* G = &s.gangs[g];
  volatile ServeSlot* slot = &s.slots[g];
  if (threadIdx.x < 2) sAbort[threadIdx.x] = 0;
  for (unsigned long long seq = 1;; seq++) {
    if (threadIdx.x == 0) {
      int stop = 0;
      const uint64_t t0 = globaltimer();
      if (leader) {
        while (true) {                                   // idle wait for the host
          if (ldVol64(&slot->seq) >= seq) break;
          if (*s.shutdown || *s.abortFlag) { stop = 1; break; }
          if (globaltimer() - t0 > s.idleTimeoutNs) { stop = 1; break; }
          __nanosleep(256);
        }
        if (!stop) {
          __threadfence_system();                        // the request was written before seq
          const volatile unsigned long long* src = (const volatile unsigned long long*)&slot->req;
          unsigned long long* dst = (unsigned long long*)&G->req;
          for (int i = 0; i < (int)(sizeof(ServeReq) / 8); i++) dst[i] = src[i];
          slot->tStart = globaltimer();
          __threadfence();
          stRelease(&G->goSeq, seq);
        } else {
          stRelease(&G->goSeq, ~0ull);
        }
      } else {
        while (true) {                                   // wait for the leader
          const uint64_t v = ldAcquire(&G->goSeq);
          if (v == ~0ull) { stop = 1; break; }
          if (v >= seq) break;
          if (globaltimer() - t0 > s.idleTimeoutNs + 2000000000ull) { stop = 1; break; }
          __nanosleep(256);
        }
      }
      sStop = stop;
      int use = 0;
      if (!stop && ((const volatile ServeReq*)&G->req)->proto == kDirect) {
        use = 2;   // the direct protocol: every CTA of the gang takes a share
      } else if (!stop) {
        const volatile ServeReq* q = (const volatile ServeReq*)&G->req;
        // a request of k vranks and C channels runs on the gang's first k x C CTAs
        use = (local < q->nranks * q->nsub) ? 1 : 0;
        ch = local / q->nranks;
        r = local % q->nranks;
        sa.nranks = q->nranks;
        if (use) {
          sa.count = q->count;
          sa.chunk = q->chunk;
          sa.slotBytes = q->slotBytes;
          sa.slotUnits = q->slotUnits;
          sa.timeoutNs = s.timeoutNs;
          sa.conns = s.conns[q->proto] + s.gangConn[g];
          sa.errClaim = s.errClaim;
          sa.err = s.err;
          sa.abortFlag = s.abortFlag;
          sa.inplaceMask = q->inplaceMask;
          sa.downOffset = 0;
          sa.coll = q->coll;
          sa.algo = kRing;
          sa.redop = q->redop;
          sa.nranks = q->nranks;
          sa.nsub = q->nsub;
          sa.root = q->root;
          sa.nsteps = s.nsteps;
          sa.upThreads = (blockDim.x / 2) / 32 * 32;
          sa.skipRank = -1;
          sa.postDiv = 0;   // serving runs sum and max only
          sa.treeNode = 1;  // and the ring only
          for (int i = 0; i < q->nranks; i++) {
            sa.send[i] = (const void*)q->send[i];
            sa.recv[i] = (void*)q->recv[i];
          }
        }
      }
      sUse = use;
      sCh = ch;
      sR = r;
    }
    __syncthreads();
    if (sStop) return;
    ch = sCh;
    r = sR;
    if (sUse == 2) {
      dispatchDirect(&G->req, (unsigned long long)local, nctas);
    } else if (sUse) {
      const int proto = sa.coll == kCopy ? kSimple : ((const volatile ServeReq*)&G->req)->proto;
      const int dtype = ((const volatile ServeReq*)&G->req)->dtype;
      const bool bytes = (sa.coll == kAllGather || sa.coll == kBroadcast ||
                          (sa.coll == kCopy && dtype < 0));
      dispatchOp(sa, proto, dtype, bytes, r, ch, &ws);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();
      atomicAdd(&G->arrive, 1ull);
      if (leader) {
        const uint64_t t0 = globaltimer();
        bool ok = true;
        while (ldAcquire(&G->arrive) < seq * nctas) {
          if (globaltimer() - t0 > s.timeoutNs) { ok = false; break; }
        }
        const int failed = (!ok || sAbort[0] || sAbort[1] || *s.errClaim) ? 1 : 0;
        slot->tEnd = globaltimer();
        if (failed) slot->err = 1;
        __threadfence_system();
        slot->done = seq;
        __threadfence_system();
        if (failed) stRelease(&G->goSeq, ~0ull);
        sStop = failed;
      } else {
        sStop = (sAbort[0] || sAbort[1]) ? 1 : 0;
      }
    }
    __syncthreads();
    if (sStop) return;
  }
}

const void* batchKernel() { return (const void*)kBatch; }
const void* serveKernel() { return (const void*)kServe; }

}  // namespace vc
