// vcomm_cluster.cuh -- the cluster protocol: LL lines in distributed shared
// memory, for latency-bound (small) collectives.
//
// One thread-block cluster per channel holds all k vranks of that channel
// (CTA r of the cluster is vrank r), so every FIFO can live in the shared
// memory of its RECEIVER: the sender stores LL lines -- 4 data bytes + a
// 4-byte flag in one 8-byte store, as in the LL protocol of Sec. III-B --
// straight into the receiver's SMEM through the cluster's distributed shared
// memory, and the receiver polls its own SMEM.  Nothing crosses L2 or the
// die-to-die link.  The step tables (Sched) and the reductions are the ones
// the other protocols use; only the FIFO medium differs.
//
// No block-wide barrier per step: every warp walks the step table on its own.
// Line pair p of a FIFO step belongs to one thread of the group, so a warp
// needs nothing from the other warps; the pair-to-thread map rotates by the
// warps each step uses, so that a small step goes to a warp that is already
// waiting for it while the previous step's warp finishes its bookkeeping.  Credits are counted in line pairs
// per slot: after reading a step, each warp adds the number of pairs it read
// to the sender's counter for that slot (a remote red.add); the sender may
// refill the slot once the counter holds every pair of every earlier use.
// Counting per slot keeps a fast warp's later steps from standing in for a
// slow warp's earlier one (a slot is reused only after its counter is full).
//
// SMEM of one CTA: kCIn incoming FIFOs of kCSlots slots of kCSlotBytes, then
// kCOut x kCSlots credit counters (one set per outgoing connection: 0 = ring
// successor or tree parent, 1 / 2 = tree children).  Incoming FIFO 0/1 = from
// tree children (or the ring predecessor in 0), 2 = from the tree parent.
// Everything starts at zero in every launch (flags are step + 1 from 0),
// behind a cluster barrier; a second cluster barrier keeps every CTA alive
// until no peer can touch its SMEM.
#pragma once
#include "vcomm_device.cuh"

namespace vc {

constexpr int kCSlots = 4;                 // slots per incoming FIFO
constexpr int kCSlotBytes = 8192;          // LL lines: 4096 data bytes per slot
constexpr int kCIn = 3;                    // incoming FIFOs per CTA
constexpr int kCOut = 3;                   // outgoing connections per CTA (credit sets)
constexpr int kCCreditOff = kCIn * kCSlots * kCSlotBytes;
constexpr int kCSmemBytes = kCCreditOff + 256;
static_assert(kCOut * kCSlots * 4 <= 256, "credit counters");
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
VDEV void redRemoteAdd(uint32_t addr, uint32_t v) {
  asm volatile("red.relaxed.cluster.shared::cluster.add.u32 [%0], %1;" ::"r"(addr), "r"(v) : "memory");
}
VDEV void ldLocal2(uint32_t addr, uint64_t& a, uint64_t& b) {
  asm volatile("ld.relaxed.cluster.shared::cta.v2.u64 {%0, %1}, [%2];" : "=l"(a), "=l"(b) : "r"(addr)
               : "memory");
}
VDEV uint32_t ldLocal(uint32_t addr) {
  uint32_t v;
  asm volatile("ld.relaxed.cluster.shared::cta.u32 %0, [%1];" : "=r"(v) : "r"(addr) : "memory");
  return v;
}
VDEV void clusterSync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::
                   : "memory");
}

// One FIFO connection as seen by one end.
struct CLink {
  int peer = -1;   // the other end's CTA rank in the cluster (-1: none)
  int fifo = 0;    // the incoming FIFO index at the receiver
  int cset = 0;    // the credit set index at the sender
};

// expected credit of slot j (registers, no dynamic indexing)
struct SlotCount {
  uint32_t c0 = 0, c1 = 0, c2 = 0, c3 = 0;
  VDEV uint32_t get(int j) const { return j == 0 ? c0 : j == 1 ? c1 : j == 2 ? c2 : c3; }
  VDEV void add(int j, uint32_t v) {
    if (j == 0) c0 += v;
    else if (j == 1) c1 += v;
    else if (j == 2) c2 += v;
    else c3 += v;
  }
};
static_assert(kCSlots == 4, "SlotCount holds four slots");

template <class T, class Op>
struct ClusterPrims {
  const KernArgs& a;
  int tid = 0, nthr = 0;
  volatile int* sAbort = nullptr;
  int rank = 0, ch = 0;
  uint32_t base = 0;           // this CTA's SMEM base (shared window address)
  int nrc = 0, nsc = 0;        // receive / send links in use (0..2)
  CLink rA, rB;                // receive links (peer = sender)
  CLink sA, sB;                // send links (peer = receiver)
  SlotCount exA, exB;          // pairs the receivers must have read per slot
  uint32_t rstep = 0, sstep = 0;
  int woff = 0;                // first warp of the current step's pairs

  VDEV uint32_t fifoAddr(int fifo, uint32_t step) const {
    return base + (uint32_t)((fifo * kCSlots + (int)(step % kCSlots)) * kCSlotBytes);
  }
  VDEV uint32_t creditAddr(int cset, int slot) const {
    return base + (uint32_t)(kCCreditOff + (cset * kCSlots + slot) * 4);
  }

  // spin until my credit counter (cset, slot) reaches `need`.  The clock is
  // first read after 256 polls: a wait that ends sooner (the usual case)
  // pays nothing for its deadline.
  VDEV bool waitCredit(int cset, int slot, uint32_t need) {
    const uint32_t ad = creditAddr(cset, slot);
    uint64_t t0 = 0;
    unsigned it = 0;
    while (ldLocal(ad) < need) {
      if (((++it) & 255u) == 0) {
        if (t0 == 0) t0 = globaltimer();
        if (*sAbort) return false;
        if (*(volatile int*)a.errClaim) return false;   // another CTA failed first
        if (*a.abortFlag) { reportFailure(a, vAborted, rank, ch, 2); return false; }
        if (globaltimer() - t0 > a.timeoutNs) { reportFailure(a, vTimeout, rank, ch, 2); return false; }
      }
    }
    return true;
  }

  // poll an LL line pair in my own SMEM until both flags equal `flag`
  // (deadline clock read lazily, as above)
  VDEV bool pollPair(uint32_t ad, uint32_t flag, uint64_t& x, uint64_t& y) {
    uint64_t t0 = 0;
    unsigned it = 0;
    while (true) {
      ldLocal2(ad, x, y);
      if ((uint32_t)(x >> 32) == flag && (uint32_t)(y >> 32) == flag) return true;
      if (((++it) & 255u) == 0) {
        if (t0 == 0) t0 = globaltimer();
        if (*sAbort) return false;
        if (*(volatile int*)a.errClaim) return false;
        if (*a.abortFlag) { reportFailure(a, vAborted, rank, ch, 3); return false; }
        if (globaltimer() - t0 > a.timeoutNs) { reportFailure(a, vTimeout, rank, ch, 3); return false; }
      }
    }
  }

  // one FIFO step of m <= 4096 / sizeof(T) elements; warp-uniform result
  VDEV bool step(bool doRecv, bool doLocal, bool doSend, bool doOut, const T* local, T* out,
                 uint32_t m) {
    doRecv = doRecv && nrc > 0;   // never touch a link that does not exist
    doSend = doSend && nsc > 0;
    const uint32_t nbytes = m * (uint32_t)sizeof(T);
    const uint32_t npairs = (nbytes + 7) / 8;
    const int sslot = (int)(sstep % kCSlots);
    const int div = (std::is_same<Op, OpAvg>::value && doRecv && doLocal && doOut) ? a.postDiv : 0;
    const int nw = nthr >> 5;
    int vt = tid - woff * 32;     // my position in this step's rotated map
    if (vt < 0) vt += nthr;
    const bool warpHasPairs = (uint32_t)(vt & ~31) < npairs;   // warp-uniform
    woff += (int)((npairs + 31) / 32);
    while (woff >= nw) woff -= nw;
    bool ok = true;
    if (doSend && (uint32_t)vt < npairs && sstep >= (uint32_t)kCSlots) {
      ok = waitCredit(sA.cset, sslot, exA.get(sslot));
      if (ok && nsc > 1) ok = waitCredit(sB.cset, sslot, exB.get(sslot));
    }
    uint32_t mine = 0;   // pairs this thread read
    if (ok) {
      const uint32_t f = rstep + 1, g = sstep + 1;
      const uint32_t inA = doRecv ? fifoAddr(rA.fifo, rstep) : 0;
      const uint32_t inB = (doRecv && nrc > 1) ? fifoAddr(rB.fifo, rstep) : 0;
      const uint32_t outA = doSend ? mapRank(fifoAddr(sA.fifo, sstep), sA.peer) : 0;
      const uint32_t outB = (doSend && nsc > 1) ? mapRank(fifoAddr(sB.fifo, sstep), sB.peer) : 0;
      for (uint32_t p = vt; p < npairs; p += nthr) {
        const int valid = (int)((nbytes - 8 * p) < 8 ? (nbytes - 8 * p) : 8);
        uint64_t v = doLocal ? loadUser8<T>((const char*)local + 8ull * p, valid) : 0;
        if (doRecv) {
          uint64_t x, y;
          if (!pollPair(inA + 16 * p, f, x, y)) { ok = false; break; }
          const uint64_t w = (uint64_t)((x & 0xffffffffull) | (y << 32));
          v = doLocal ? applyWord<T, Op>(w, v) : w;
          if (nrc > 1) {
            if (!pollPair(inB + 16 * p, f, x, y)) { ok = false; break; }
            v = applyWord<T, Op>((uint64_t)((x & 0xffffffffull) | (y << 32)), v);
          }
          mine++;
        }
        if (div) v = divWord<T>(v, div);
        if (doOut) storeUser8<T>((char*)out + 8ull * p, v, valid);
        if (doSend) {
          const uint64_t lo = v & 0xffffffffull, hi = v >> 32;
          stRemote2(outA + 16 * p, lo | ((uint64_t)g << 32), hi | ((uint64_t)g << 32));
          if (nsc > 1) stRemote2(outB + 16 * p, lo | ((uint64_t)g << 32), hi | ((uint64_t)g << 32));
        }
      }
    }
    if (!ok) *sAbort = 1;
    // one warp-wide sum: the pairs read, plus 2^20 per failed lane, so the
    // whole warp agrees before anyone returns a slot or moves on (a warp
    // without pairs in this step neither waited nor read)
    const uint32_t w =
        warpHasPairs ? __reduce_add_sync(0xffffffffu, mine + (ok ? 0u : (1u << 20))) : 0u;
    if (w >= (1u << 20)) return false;
    if (doRecv) {
      if ((threadIdx.x & 31) == 0 && w) {
        const int rslot = (int)(rstep % kCSlots);
        redRemoteAdd(mapRank(creditAddr(rA.cset, rslot), rA.peer), w);
        if (nrc > 1) redRemoteAdd(mapRank(creditAddr(rB.cset, rslot), rB.peer), w);
      }
      rstep++;
    }
    if (doSend) {
      exA.add(sslot, npairs);
      exB.add(sslot, npairs);
      sstep++;
    }
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
  // zero my FIFOs and credit counters, then nobody writes into anybody
  // before everybody has zeroed
  {
    uint4* z = (uint4*)smem;
    for (int i = threadIdx.x; i < kCSmemBytes / 16; i += blockDim.x) z[i] = make_uint4(0, 0, 0, 0);
  }
  __syncthreads();
  clusterSync();
  const bool skip = (r == a.skipRank);   // injected fault: take no part, keep the barriers
  if (!skip) {
    ClusterPrims<T, Op> pr{a};
    pr.tid = threadIdx.x;
    pr.nthr = blockDim.x;
    pr.sAbort = sAbort;
    pr.rank = r;
    pr.ch = ch;
    pr.base = smemAddr(smem);
    int role = kRoleRing;
    bool leaf = false;
    if (a.algo == kTree) {
      const int t = ch & 1;
      int parent, c0, c1;
      treeLinksM(k, a.treeNode, t, r, &parent, &c0, &c1);
      leaf = (c0 < 0);
      // credit sets at a sender: 0 = its up link, 1 / 2 = its down links to
      // child0 / child1.  Incoming FIFOs: 0 / 1 = from child0 / child1, 2 =
      // from the parent.
      CLink fromC0{c0, 0, 0}, fromC1{c1, 1, 0};
      CLink toC0{c0, 2, 1}, toC1{c1, 2, 2};
      if (parent < 0 || (int)threadIdx.x < a.upThreads) {
        role = parent < 0 ? kRoleTreeRoot : kRoleTreeUp;
        if (c0 >= 0) { (pr.nrc == 0 ? pr.rA : pr.rB) = fromC0; pr.nrc++; }
        if (c1 >= 0) { (pr.nrc == 0 ? pr.rA : pr.rB) = fromC1; pr.nrc++; }
        if (parent < 0) {
          if (c0 >= 0) { (pr.nsc == 0 ? pr.sA : pr.sB) = toC0; pr.nsc++; }
          if (c1 >= 0) { (pr.nsc == 0 ? pr.sA : pr.sB) = toC1; pr.nsc++; }
        } else {
          int p0, pc0, pc1;
          treeLinksM(k, a.treeNode, t, parent, &p0, &pc0, &pc1);
          pr.sA = CLink{parent, (pc0 == r) ? 0 : 1, 0};
          pr.nsc = 1;
          pr.nthr = a.upThreads;
        }
      } else {
        role = kRoleTreeDown;
        pr.tid = threadIdx.x - a.upThreads;
        pr.nthr = blockDim.x - a.upThreads;
        pr.sAbort = sAbort + 1;
        int p0, pc0, pc1;
        treeLinksM(k, a.treeNode, t, parent, &p0, &pc0, &pc1);
        pr.rA = CLink{parent, 2, (pc0 == r) ? 1 : 2};
        pr.nrc = 1;
        if (c0 >= 0) { (pr.nsc == 0 ? pr.sA : pr.sB) = toC0; pr.nsc++; }
        if (c1 >= 0) { (pr.nsc == 0 ? pr.sA : pr.sB) = toC1; pr.nsc++; }
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
      if (hasSend) { pr.sA = CLink{modk(r + 1, k), 0, 0}; pr.nsc = 1; }
      if (hasRecv) { pr.rA = CLink{modk(r - 1, k), 0, 0}; pr.nrc = 1; }
    }
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
