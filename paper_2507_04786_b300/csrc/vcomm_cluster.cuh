// vcomm_cluster.cuh -- the cluster protocol: LL lines in distributed shared
// memory, for latency-bound (small) collectives.
//
// One thread-block cluster per channel holds all k vranks of that channel
// (CTA r of the cluster is vrank r), so every FIFO can live in the shared
// memory of its RECEIVER: the sender stores LL lines -- 4 data bytes + a
// 4-byte flag in one 8-byte store, as in the LL protocol of Sec. III-B --
// straight into the receiver's SMEM through the cluster's distributed shared
// memory, the receiver polls its own SMEM, and the receiver returns credits by
// storing its consumed-step count into the sender's SMEM.  Nothing crosses L2
// or the die-to-die link, so a hop costs a DSMEM store instead of two L2
// round trips.  The step tables (Sched) and the reductions are the ones the
// other protocols use; only the FIFO medium differs.
//
// SMEM of one CTA: kCIn incoming FIFOs of kCSlots slots of kCSlotBytes, then
// kCIn credit words (the heads of this CTA's outgoing connections, written by
// their receivers).  Incoming FIFO 0/1 = from tree children (or the ring
// predecessor in 0), 2 = from the tree parent.  Everything starts at zero in
// every launch (flags are step + 1 from 0), behind a cluster barrier; a second
// cluster barrier keeps every CTA alive until no peer can touch its SMEM.
#pragma once
#include "vcomm_device.cuh"

namespace vc {

constexpr int kCSlots = 4;                 // slots per incoming FIFO
constexpr int kCSlotBytes = 8192;          // LL lines: 4096 data bytes per slot
constexpr int kCIn = 3;                    // incoming FIFOs per CTA
constexpr int kCSmemBytes = kCIn * kCSlots * kCSlotBytes + 256;
static_assert(kCSmemBytes == 3 * 4 * 8192 + 256, "update kClusterSmemBytes in vcomm_kernels.h");

VDEV uint32_t smemAddr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
// address of the same SMEM offset in CTA `rank` of the cluster
VDEV uint32_t mapRank(uint32_t addr, int rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(addr), "r"(rank));
  return r;
}
VDEV void stRemote2(uint32_t addr, uint64_t a, uint64_t b) {
  asm volatile("st.relaxed.cluster.shared::cluster.v2.u64 [%0], {%1, %2};" ::"r"(addr), "l"(a), "l"(b)
               : "memory");
}
VDEV void stRemoteRelease(uint32_t addr, uint64_t v) {
  asm volatile("st.release.cluster.shared::cluster.u64 [%0], %1;" ::"r"(addr), "l"(v) : "memory");
}
VDEV void ldLocal2(uint32_t addr, uint64_t& a, uint64_t& b) {
  asm volatile("ld.relaxed.cluster.shared::cta.v2.u64 {%0, %1}, [%2];" : "=l"(a), "=l"(b) : "r"(addr)
               : "memory");
}
VDEV uint64_t ldLocalAcquire(uint32_t addr) {
  uint64_t v;
  asm volatile("ld.acquire.cluster.shared::cta.u64 %0, [%1];" : "=l"(v) : "r"(addr) : "memory");
  return v;
}
VDEV void clusterSync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::
                   : "memory");
}

// A connection seen from one end: the peer's CTA rank and the FIFO index
// at the receiver.
struct CLink {
  int peer;    // -1: none
  int fifo;    // receiver-side incoming FIFO index
};

template <class T, class Op>
struct ClusterPrims {
  const KernArgs& a;
  int tid, nthr, barId;
  volatile int* sAbort;
  int rank, ch;
  uint32_t base;               // this CTA's SMEM base (shared window address)
  int nrc, nsc;
  int rf[2];                   // my incoming FIFO indices (receives)
  CLink sl[2];                 // my outgoing links (sends)
  int cr[2];                   // my credit-word index per outgoing link
  int rpeer[2];                // the sender of each receive (for returning credits)
  int rcredit[2];              // the credit-word index at that sender
  uint64_t rstep[2], sstep[2];

  VDEV uint32_t fifoAddr(int fifo, uint64_t step) const {
    return base + (uint32_t)((fifo * kCSlots + (int)(step % kCSlots)) * kCSlotBytes);
  }
  VDEV uint32_t creditAddr(int i) const { return base + (uint32_t)(kCIn * kCSlots * kCSlotBytes + 8 * i); }
  VDEV void bar() { groupBar(barId, nthr); }

  // thread 0 waits until the receiver has freed slot `step` of link i
  VDEV bool waitCredit(int i, uint64_t step) {
    if (step + 1 <= (uint64_t)kCSlots) return true;
    const uint64_t need = step + 1 - kCSlots;
    const uint32_t ad = creditAddr(cr[i]);
    if (ldLocalAcquire(ad) >= need) return true;
    const uint64_t t0 = globaltimer();
    unsigned it = 0;
    while (ldLocalAcquire(ad) < need) {
      if (((++it) & 255u) == 0) {
        if (*(volatile int*)a.errClaim) return false;   // another CTA failed first
        if (*a.abortFlag) { reportFailure(a, vAborted, rank, ch, 2); return false; }
        if (globaltimer() - t0 > a.timeoutNs) { reportFailure(a, vTimeout, rank, ch, 2); return false; }
      }
    }
    return true;
  }

  // poll an LL line pair in my own SMEM until both flags equal `flag`
  VDEV bool pollPair(uint32_t ad, uint32_t flag, uint64_t& x, uint64_t& y) {
    ldLocal2(ad, x, y);
    if ((uint32_t)(x >> 32) == flag && (uint32_t)(y >> 32) == flag) return true;
    const uint64_t t0 = globaltimer();
    unsigned it = 0;
    while (true) {
      ldLocal2(ad, x, y);
      if ((uint32_t)(x >> 32) == flag && (uint32_t)(y >> 32) == flag) return true;
      if (((++it) & 255u) == 0) {
        if (*sAbort) return false;
        if (*(volatile int*)a.errClaim) { *sAbort = 1; return false; }
        if (*a.abortFlag) { reportFailure(a, vAborted, rank, ch, 3); *sAbort = 1; return false; }
        if (globaltimer() - t0 > a.timeoutNs) { reportFailure(a, vTimeout, rank, ch, 3); *sAbort = 1; return false; }
      }
    }
  }

  VDEV bool step(bool doRecv, bool doLocal, bool doSend, bool doOut, const T* local, T* out,
                 uint32_t m) {
    doRecv = doRecv && nrc > 0;   // never touch a link that does not exist
    doSend = doSend && nsc > 0;
    if (tid == 0 && doSend) {
      bool ok = waitCredit(0, sstep[0]);
      if (ok && nsc > 1) ok = waitCredit(1, sstep[1]);
      if (!ok) *sAbort = 1;
    }
    bar();
    if (*sAbort) return false;
    const uint32_t nbytes = m * (uint32_t)sizeof(T);
    const uint32_t npairs = (nbytes + 7) / 8;
    const uint32_t f0 = (uint32_t)(rstep[0] + 1), f1 = (uint32_t)(rstep[1] + 1);
    const uint32_t g0 = (uint32_t)(sstep[0] + 1), g1 = (uint32_t)(sstep[1] + 1);
    const uint32_t in0 = doRecv ? fifoAddr(rf[0], rstep[0]) : 0;
    const uint32_t in1 = (doRecv && nrc > 1) ? fifoAddr(rf[1], rstep[1]) : 0;
    const uint32_t out0 = doSend ? mapRank(fifoAddr(sl[0].fifo, sstep[0]), sl[0].peer) : 0;
    const uint32_t out1 = (doSend && nsc > 1) ? mapRank(fifoAddr(sl[1].fifo, sstep[1]), sl[1].peer) : 0;
    for (uint32_t p = tid; p < npairs; p += nthr) {
      const int valid = (int)((nbytes - 8 * p) < 8 ? (nbytes - 8 * p) : 8);
      uint64_t v = doLocal ? loadUser8<T>((const char*)local + 8ull * p, valid) : 0;
      bool fail = false;
      if (doRecv) {
        uint64_t x, y;
        if (!pollPair(in0 + 16 * p, f0, x, y)) { fail = true; }
        else {
          const uint64_t w = (uint64_t)((x & 0xffffffffull) | (y << 32));
          v = doLocal ? applyWord<T, Op>(w, v) : w;
          if (nrc > 1) {
            if (!pollPair(in1 + 16 * p, f1, x, y)) fail = true;
            else v = applyWord<T, Op>((uint64_t)((x & 0xffffffffull) | (y << 32)), v);
          }
        }
      }
      if (fail) break;
      if (doOut) storeUser8<T>((char*)out + 8ull * p, v, valid);
      if (doSend) {
        const uint64_t lo = v & 0xffffffffull, hi = v >> 32;
        stRemote2(out0 + 16 * p, lo | ((uint64_t)g0 << 32), hi | ((uint64_t)g0 << 32));
        if (nsc > 1) stRemote2(out1 + 16 * p, lo | ((uint64_t)g1 << 32), hi | ((uint64_t)g1 << 32));
      }
    }
    bar();
    if (*sAbort) return false;
    if (tid == 0 && doRecv) {   // return the slots: the readers are done
      stRemoteRelease(mapRank(creditAddr(rcredit[0]), rpeer[0]), rstep[0] + 1);
      if (nrc > 1) stRemoteRelease(mapRank(creditAddr(rcredit[1]), rpeer[1]), rstep[1] + 1);
    }
    if (doSend) { sstep[0]++; sstep[1]++; }
    if (doRecv) { rstep[0]++; rstep[1]++; }
    return true;
  }

  VDEV bool run(bool doRecv, bool doLocal, bool doSend, bool doOut, const T* local, T* out,
                unsigned long long n) {
    const unsigned long long cap = (kCSlotBytes / 2) / sizeof(T);
    unsigned long long done = 0;
    while (done < n) {
      unsigned long long m = n - done;
      if (m > cap) m = cap;
      if (!step(doRecv, doLocal, doSend, doOut, local + done, out + done, (uint32_t)m)) return false;
      done += m;
    }
    return true;
  }
};

// CTA (r, ch) of a cluster-protocol launch; the cluster is channel ch.
template <class T, class Op>
VDEV void runClusterWorker(const KernArgs& a, int r, int ch, volatile int* sAbort, unsigned char* smem) {
  const int k = a.nranks;
  // zero my FIFOs and credit words, then nobody writes into anybody before
  // everybody has zeroed
  {
    uint4* z = (uint4*)smem;
    for (int i = threadIdx.x; i < kCSmemBytes / 16; i += blockDim.x) z[i] = make_uint4(0, 0, 0, 0);
  }
  __syncthreads();
  clusterSync();
  const bool skip = (r == a.skipRank);   // injected fault: take no part, keep the barriers
  if (!skip) {
    int tid = threadIdx.x, nthr = blockDim.x, barId = 0, role = kRoleRing;
    bool leaf = false;
    volatile int* ab = sAbort;
    ClusterPrims<T, Op> pr{a, 0, 0, 0, nullptr, r, ch, smemAddr(smem), 0, 0};
    pr.rstep[0] = pr.rstep[1] = pr.sstep[0] = pr.sstep[1] = 0;
    if (a.algo == kTree) {
      const int t = ch & 1;
      int parent, c0, c1;
      treeLinks(k, t, r, &parent, &c0, &c1);
      leaf = (c0 < 0);
      // my position among my parent's children (its incoming FIFO 0 or 1)
      int upFifo = 0;
      if (parent >= 0) {
        int p0, pc0, pc1;
        treeLinks(k, t, parent, &p0, &pc0, &pc1);
        upFifo = (pc0 == r) ? 0 : 1;
      }
      // credit words (heads of MY outgoing links, written by their receivers):
      // 0 = my up link, 1 / 2 = my down links to child0 / child1
      if (parent < 0 || (int)threadIdx.x < a.upThreads) {
        role = parent < 0 ? kRoleTreeRoot : kRoleTreeUp;
        // receive from the children: child0 into FIFO 0, child1 into FIFO 1;
        // their up links are credited in each child's word 0
        if (c0 >= 0) { pr.rf[pr.nrc] = 0; pr.rpeer[pr.nrc] = c0; pr.rcredit[pr.nrc] = 0; pr.nrc++; }
        if (c1 >= 0) { pr.rf[pr.nrc] = 1; pr.rpeer[pr.nrc] = c1; pr.rcredit[pr.nrc] = 0; pr.nrc++; }
        if (parent < 0) {   // the root sends down to its children's FIFO 2
          if (c0 >= 0) { pr.sl[pr.nsc] = CLink{c0, 2}; pr.cr[pr.nsc] = 1; pr.nsc++; }
          if (c1 >= 0) { pr.sl[pr.nsc] = CLink{c1, 2}; pr.cr[pr.nsc] = 2; pr.nsc++; }
        } else {            // the up group sends to the parent
          pr.sl[0] = CLink{parent, upFifo};
          pr.cr[0] = 0;
          pr.nsc = 1;
          nthr = a.upThreads;
          barId = 1;
        }
      } else {
        role = kRoleTreeDown;
        tid = threadIdx.x - a.upThreads;
        nthr = blockDim.x - a.upThreads;
        barId = 2;
        ab = sAbort + 1;
        // receive from the parent into FIFO 2; credit the parent's word for
        // its link to me (1 if I am its child0, else 2)
        int p0, pc0, pc1;
        treeLinks(k, t, parent, &p0, &pc0, &pc1);
        pr.rf[0] = 2;
        pr.rpeer[0] = parent;
        pr.rcredit[0] = (pc0 == r) ? 1 : 2;
        pr.nrc = 1;
        if (c0 >= 0) { pr.sl[pr.nsc] = CLink{c0, 2}; pr.cr[pr.nsc] = 1; pr.nsc++; }
        if (c1 >= 0) { pr.sl[pr.nsc] = CLink{c1, 2}; pr.cr[pr.nsc] = 2; pr.nsc++; }
      }
    } else {
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
      if (hasSend) { pr.sl[0] = CLink{modk(r + 1, k), 0}; pr.cr[0] = 0; pr.nsc = 1; }
      if (hasRecv) { pr.rf[0] = 0; pr.rpeer[0] = modk(r - 1, k); pr.rcredit[0] = 0; pr.nrc = 1; }
    }
    pr.tid = tid;
    pr.nthr = nthr;
    pr.barId = barId;
    pr.sAbort = ab;
    Sched sc;
    sc.init(a, r, ch, role, leaf, (int)sizeof(T));
    const T* x = (const T*)a.send[r];
    T* y = (T*)a.recv[r];
    Desc d;
    while (sc.next(d, (int)sizeof(T))) {
      if (!pr.run(d.recv, d.local, d.send, d.out, x + d.lo, y + d.oo, d.n)) break;
    }
  }
  // nobody leaves while a peer may still store into its SMEM
  __syncthreads();
  clusterSync();
}

}  // namespace vc
