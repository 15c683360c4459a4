// vcomm_internal.h -- structures shared by the host runtime and the kernels.
//
// Layout of a communicator's device state (all in one GPU's HBM):
//   * per (algorithm, protocol) one FIFO arena: nconn connections, each a ring
//     of `nsteps` slots of `slotBytes` (Sec. V-C, Table "NCCL channel buffer
//     sizes"), plus two 128-byte counter lines per connection: `tail` (FIFO
//     steps the sender has posted) and `head` (steps the receiver has
//     consumed), the head/tail pair of the paper's P2P transport (Sec. IV-A).
//   * ring connections: index ch * k + r is the edge r -> r+1 of channel ch.
//   * tree connections: sub-channel j (two per channel), index j * k + r is the
//     up edge r -> parent(r); index downOffset + j * k + r the down edge
//     parent(r) -> r, with downOffset = (2 x the communicator's channels) x k.
#pragma once
#include <algorithm>
#include <stddef.h>
#include <stdint.h>

#include "vcomm.h"

#if defined(__CUDACC__)
#define VC_HD __host__ __device__ __forceinline__
#else
#define VC_HD inline
#endif

namespace vc {

enum Coll : int { kAllReduce = 0, kReduceScatter = 1, kAllGather = 2, kBroadcast = 3, kReduce = 4,
                  kCopy = 5 };
enum Algo : int { kRing = 0, kTree = 1 };
enum Proto : int { kSimple = 0, kLL = 1, kLL128 = 2, kCluster = 3, kDirect = 4 };
enum DType : int { kI32 = 0, kF32 = 1, kF16 = 2, kBF16 = 3, kI8 = 4, kU8 = 5, kU32 = 6, kI64 = 7,
                   kU64 = 8, kF64 = 9 };
constexpr int kNumDtypes = 10;
// element-wise ops of the kernels; avg adds like kSum and divides by
// KernArgs::postDiv in the step that completes a value (its own kernels, so
// that the other reductions compile without that step)
enum OpKind : int { kSum = 0, kMax = 1, kProd = 2, kMin = 3, kAvg = 4 };
constexpr int kNumOps = 5;

constexpr int kCounterStride = 16;

// Largest CTA each protocol's kernels are compiled for; the register budget
// per thread is 65536 / that.  Every protocol takes 512 threads and 128
// registers: Simple and LL128 stream 16-byte vectors with several loads in
// flight per thread, and LL keeps four line pairs per thread in flight (at
// 1024 threads its 64 registers spilled on the step path: 8 x 256 MiB ring
// AllReduce 5.97 -> 3.53 ms, small calls 5-21 % faster at 512).  A
// cluster-protocol FIFO step is at most 512 line pairs: one per thread.
constexpr int maxThreadsFor(int) { return 512; }

struct ConnDev {
  char* buf;                       // nsteps slots of slotBytes
  unsigned long long* tail;        // written only by the sending CTA
  unsigned long long* head;        // written only by the receiving CTA
  unsigned long long unused;
};

// first device-side failure; lives in host-mapped memory so that the host can
// read it without synchronising
struct ErrWord {
  int code;      // vResult_t
  int rank;
  int channel;
  int where;     // 1 = wait on tail, 2 = wait on head (credit), 3 = LL/LL128 line poll,
                 // 4 = a bulk copy into shared memory, 5 = a misaligned staged buffer
};

struct KernArgs {
  const void* send[VCOMM_MAX_RANKS];
  void* recv[VCOMM_MAX_RANKS];
  unsigned long long count;        // units partitioned over channels
  unsigned long long chunk;        // chunkCount in units (multiple of a 16-byte pack)
  unsigned long long slotBytes;    // bytes of one FIFO slot
  unsigned long long slotUnits;    // data units one FIFO slot carries
  unsigned long long timeoutNs;    // deadline of every flag wait
  ConnDev* conns;
  int* errClaim;                   // device word: first failure claims it
  ErrWord* err;                    // host-mapped report
  const volatile int* abortFlag;   // host-mapped abort word
  unsigned long long inplaceMask;  // bit r: rank r runs in place
  unsigned long long downOffset;   // tree: index of the first down connection
  int coll;
  int algo;
  int redop;                       // OpKind (read by the batch kernel's dispatch)
  int nranks;
  int nsub;                        // CTAs per rank: channels (ring) or 2 x channels (tree)
  int root;
  int nsteps;
  int upThreads;                   // tree: threads of the reduce (up) group on non-root ranks
  int skipRank;                    // fault injection: this vrank's CTAs return at once (-1: none)
  int postDiv;                     // avg: the step that completes a value divides it by this (0: none)
  int treeNode;                    // tree: vranks per node of the hierarchical tree (0 or 1: flat)
};

// ---- batched launch: many collectives in one persistent kernel (group calls,
// Sec. II-A-4).  The grid is `ngangs` gangs of nranks x cpg CTAs; gang g runs
// its ops one after another on channels [g * cpg, (g + 1) * cpg) of the
// communicator's arenas.  The whole description travels as one kernel
// parameter (< 32 KB), so a CUDA graph that captured the launch needs no host
// buffer at replay time.
constexpr int kMaxBatchOps = 64;
constexpr int kMaxBatchPtrs = 2048;   // send + recv pointers of all ops
constexpr int kMaxGangs = 8;

struct BatchOpDesc {
  unsigned long long count, chunk, slotBytes, slotUnits, inplaceMask, downOffset;
  const ConnDev* conns;              // the (algo, proto) arena, before the gang offset
  int coll, algo, proto, dtype, redop, nsub, root, ptrBase;  // ptrs[ptrBase..+k) send, then recv
  int postDiv, pad;
};

struct BatchArgs {
  unsigned long long timeoutNs;
  int* errClaim;
  ErrWord* err;
  const volatile int* abortFlag;
  int nops, nranks, ngangs, cpg, nsteps, treeNode;
  int gangStart[kMaxGangs + 1];      // gang g runs order[gangStart[g] .. gangStart[g+1])
  unsigned char order[kMaxBatchOps];
  BatchOpDesc ops[kMaxBatchOps];
  const void* ptrs[kMaxBatchPtrs];
};

// ---- serving: a persistent kernel whose gangs take requests from host-mapped
// mailboxes (continuous batching).  Gang g owns CTAs [gangCta[g], gangCta[g+1])
// laid out as gangCpg[g] channels x kmax vranks and ring connections
// [gangConn[g], gangConn[g] + gangCpg[g] * kmax) of each protocol arena.
constexpr int kServeMaxRanks = 16;
constexpr int kMaxServeGangs = 16;

struct ServeReq {
  int coll, proto, dtype, redop, nranks, nsub, root;
  int vec;                           // direct protocol: as DirectArgs::vec
  unsigned long long count, chunk, slotUnits, slotBytes, inplaceMask;
  const void* send[kServeMaxRanks];
  void* recv[kServeMaxRanks];
};

struct ServeSlot {                   // host-mapped mailbox of one gang
  unsigned long long seq;            // host: requests posted so far
  unsigned long long done;           // device: requests completed so far
  unsigned long long tStart, tEnd;   // device %globaltimer of the last request
  unsigned long long err;            // device: nonzero once the gang stopped on a failure
  unsigned long long pad[3];
  ServeReq req;                      // the posted request (valid while seq > done)
};

struct ServeGang {                   // device memory, one per gang
  unsigned long long goSeq;          // leader -> gang: request `goSeq` is in req (~0: stop)
  unsigned long long pad0[15];
  unsigned long long arrive;         // gang barrier: CTAs that finished, cumulative
  unsigned long long pad1[15];
  ServeReq req;
};

struct ServeArgs {
  ServeSlot* slots;
  ServeGang* gangs;
  const volatile int* shutdown;      // host-mapped
  int* errClaim;
  ErrWord* err;
  const volatile int* abortFlag;
  unsigned long long timeoutNs, idleTimeoutNs;
  ConnDev* conns[3];                 // ring arena per protocol
  int ngangs, kmax, nsteps, pad;
  int gangCta[kMaxServeGangs + 1];
  int gangCpg[kMaxServeGangs];
  int gangConn[kMaxServeGangs];
};

// ---- serving mode 3 ("tiles"): one resident kernel for direct-protocol
// requests.  CTA 0 ingests requests from a host-mapped ring (in order) into
// device state and publishes them on one of two device queues (small
// requests, then large ones); every other CTA takes the next tile (a range of
// 16-byte units) of the first request in the small queue that has tiles left,
// else of the large queue; the CTA that finishes a request's last tile writes
// its completion into host-mapped memory.  Requests never wait on each other.
constexpr int kTileRing = 4096;        // request ring entries

struct TileReq {                       // host-mapped ring entry, written by the host
  ServeReq req;                        // a direct-protocol request (proto == kDirect)
  // staged requests (16-byte aligned): tiles are byte ranges of one block
  // (AllReduce: the buffer; ReduceScatter / AllGather: block b of k) that
  // move by bulk copies; otherwise tiles are ranges of the register kernels'
  // units (elements, or bytes for AllGather)
  unsigned long long staged;           // 1: bulk-copy tiles
  unsigned long long units;            // register path: units of all blocks
  unsigned long long tileUnits;        // register path: units per tile
  unsigned long long blockBytes;       // staged: 16-byte units of one block, in bytes
  unsigned long long tileBytes;        // staged: bytes of a block per tile (a multiple of 16)
  unsigned long long perBlock;         // staged: tiles per block
  unsigned long long ntiles;           // >= 1 (the last tile also does the element tails)
  unsigned long long klass;            // 0: small (served first), 1: large
  unsigned long long seq;              // written last: the request's sequence number + 1
  unsigned long long pad[7];
};

struct TileDone {                      // host-mapped, one per ring entry, written by the device
  unsigned long long seq;              // sequence number + 1 of the completed request
  unsigned long long tStart, tEnd;     // %globaltimer at ingest and at completion
  unsigned long long pad;
};

struct TileCtl {                       // host-mapped control words
  unsigned long long ingested;         // device: requests ingested so far (a sequence number)
  unsigned long long completed;        // device: requests completed so far
  int shutdown;                        // host: stop after the ingested requests
  int error;                           // device: a bulk copy did not complete in time (vTimeout)
  int stopped;                         // device: the kernel has stopped taking work
  int pad;
};

struct TileState {                     // device memory, one per ring entry
  ServeReq req;                        // copied from the ring entry with staged .. klass
  unsigned long long staged, units, tileUnits, blockBytes, tileBytes, perBlock, ntiles, klass;
  unsigned long long next;             // tiles claimed (atomic; may run past ntiles)
  unsigned long long pad0[7];
  unsigned long long done;             // tiles finished (atomic)
  unsigned long long pad1[7];
  unsigned long long seq, tStart;
};

struct TileQueues {                    // device memory, zeroed before the first launch
  unsigned long long tail[2];          // requests published per class (the ingester only)
  unsigned long long urgent;           // the ingester: the large queue's head has waited too long
  unsigned long long pad0[13];
  unsigned long long head[2];          // first entry per class that may still have tiles
  unsigned long long pad1[14];
  unsigned long long completed;        // requests completed (atomic)
  unsigned long long pad2[15];
  int stop;                            // ingester -> workers
  int pad3[31];
  unsigned long long entry[2][kTileRing];   // (position << 32) | (ring entry + 1)
};

struct TileArgs {
  TileReq* ring;                       // host-mapped
  TileDone* done;                      // host-mapped
  TileCtl* ctl;                        // host-mapped
  TileState* state;
  TileQueues* q;
  unsigned long long firstSeq;         // the first request this launch ingests
  unsigned long long idleTimeoutNs;    // stop after this long with nothing to do
  unsigned long long drainTimeoutNs;   // shutdown: wait at most this long for work in progress
  unsigned long long copyTimeoutNs;    // a bulk copy that takes longer fails the kernel
  unsigned stageBytes;                 // shared memory per pipeline stage (a multiple of 128)
  int pad;
};

// ---- a group's direct calls as tiles of one launch (the tile engine of the
// serving kernel over a fixed list: CTA j takes tiles j, j + grid, ...).
// Op i owns tiles [tileStart[i], tileStart[i + 1]); its send / recv pointers
// are ptrs[ptrBase .. + nranks) and ptrs[ptrBase + nranks .. + nranks).
struct TileOpDesc {
  unsigned long long count, chunk, inplaceMask;
  unsigned long long staged, units, tileUnits, blockBytes, tileBytes, perBlock, ntiles, tileStart;
  int coll, dtype, redop, nranks, nsub, root, vec, ptrBase;
};
// The tiles of one direct-protocol op (host side, serving and groups).
// Staged (16-byte aligned buffers; ReduceScatter / AllGather blocks that are
// not whole 16-byte units too): byte ranges of a block, whole 4 KiB pieces.
// Otherwise ranges of the register kernels' units, whole iterations (`iter` units) of
// a CTA.  About two tiles per worker CTA (`workers`), and at most
// kTileMaxTraffic bytes of traffic per tile (about 120 us of one SM's share
// of HBM) so that small work never waits long for a free CTA.
// count: elements, or bytes for AllGather / Broadcast; vec as DirectArgs::vec.
constexpr unsigned long long kTileMaxTraffic = 4ull << 20;
struct TileGeometry {
  unsigned long long staged, units, tileUnits, blockBytes, tileBytes, perBlock, ntiles;
  int vec;   // the op's DirectArgs::vec in the engine (register reductions: 0)
};
inline TileGeometry tileGeometry(int coll, int k, unsigned long long count, int esz, int vec,
                                 unsigned long long workers, unsigned long long iter, bool shared = false) {
  TileGeometry g{};
  const bool copy = (coll == kAllGather || coll == kBroadcast);
  const unsigned long long unitBytes = copy ? 1ull : (unsigned long long)esz;
  const unsigned long long blocks = (coll == kReduceScatter || coll == kAllGather) ? (unsigned long long)k : 1ull;
  // traffic per byte of a block: k inputs and k outputs (AllReduce), else k + 1
  const unsigned long long factor = coll == kAllReduce ? 2ull * k : (unsigned long long)k + 1;
  const unsigned long long twoW = 2ull * (workers > 0 ? workers : 1);
  const unsigned long long Ev = 16 / unitBytes;   // elements (bytes) per 16-byte unit
  // staged: aligned buffers of any collective, and ReduceScatter / AllGather
  // blocks that are not whole units (shifted windows: a ReduceScatter block's
  // full units; an AllGather block's aligned destination units but the last,
  // its edge bytes going with the tail)
  const bool stageable = vec == 1 || vec == 2;
  g.blockBytes = !stageable ? 0 : (vec == 2 && coll == kAllGather) ? (count >= 32 ? count / 16 * 16 - 16 : 0)
                                                                    : (count / Ev) * 16;
  g.staged = (stageable && g.blockBytes >= (vec == 2 ? 32u : 16u)) ? 1 : 0;
  if (g.staged) {
    const unsigned long long piece = 4096;
    // shared out statically (group calls): AllReduce tiles of at most 64 KiB,
    // so that the CTAs sweep neighbouring bytes of every buffer together
    // (measured 1-6 % faster than traffic-sized tiles on 4..16 vranks; with
    // tiles claimed one at a time, as in serving, the claims cost more)
    const unsigned long long cap = std::max<unsigned long long>(piece, kTileMaxTraffic / factor / piece * piece);
    const unsigned long long maxTile = (shared && coll == kAllReduce) ? std::min<unsigned long long>(cap, 64ull << 10)
                                                                        : cap;
    unsigned long long tb = (blocks * g.blockBytes + twoW - 1) / twoW;
    tb = std::min(std::max(tb, piece), maxTile);
    tb = (tb + piece - 1) / piece * piece;
    g.tileBytes = tb;
    g.perBlock = (g.blockBytes + tb - 1) / tb;
    g.ntiles = blocks * g.perBlock;
  }
  // the register path folds reductions element by element, copies as given
  g.vec = (g.staged || copy) ? vec : 0;
  if (!g.staged) {
    const unsigned long long E = g.vec ? Ev : 1;
    g.units = (g.vec == 2 && copy) ? count * blocks / 16 : (count / E) * blocks;
    const unsigned long long unitTraffic = E * unitBytes * factor;
    const unsigned long long maxTile = std::max<unsigned long long>(iter, kTileMaxTraffic / unitTraffic / iter * iter);
    unsigned long long tu = (g.units + twoW - 1) / twoW;
    tu = std::min(std::max(tu, iter), maxTile);
    tu = (tu + iter - 1) / iter * iter;
    g.tileUnits = tu;
    g.ntiles = std::max<unsigned long long>(1, (g.units + tu - 1) / tu);
  }
  return g;
}

struct TileBatchArgs {
  int nops;
  unsigned stageBytes;
  unsigned long long totalTiles;
  unsigned long long copyTimeoutNs;
  int* errClaim;
  ErrWord* err;
  TileOpDesc ops[kMaxBatchOps];
  const void* ptrs[kMaxBatchOps * 2 * kServeMaxRanks];
};

// ---- the direct protocol (no FIFO): one thread computes a unit's whole
// ring chain from the k user buffers.  count is in elements (AllReduce,
// ReduceScatter's recvcount, Reduce) or bytes (AllGather, Broadcast); chunk
// is the ring AllReduce chunkCount that fixes the segments (and so the fold
// order), nsub the channel count.
struct DirectArgs {
  const void* send[64];
  void* recv[64];
  unsigned long long count;
  unsigned long long chunk;
  unsigned long long inplaceMask;
  int coll, nranks, nsub, root;
  int vec;                         // 1: every access is a 16-byte vector; 2: 16-byte aligned
                                   // buffers, ReduceScatter / AllGather blocks that are not whole
                                   // 16-byte units (shifted vectors); 0: element accesses
  int postDiv;                     // avg: divide the folded value by this (0: none)
  // the staged reducing kernel (kDirectReduceStaged) only:
  int stages;                      // tiles of loads in flight (2 or 3)
  unsigned long long tileBytes;    // bytes of one rank's tile (multiple of 128)
  unsigned long long timeoutNs;    // deadline of every wait for a bulk copy
  int* errClaim;                   // device word: first failure claims it
  ErrWord* err;                    // host-mapped report
};

// ---- copies staged through shared memory (kCopyStaged): AllGather,
// Broadcast and point-to-point transfers as tasks.  Task i copies `bytes`
// (a multiple of 16) from `src` to dsts[dstBase + d] + dstOff for d < ndst,
// skipping the destinations whose bit is set in skipMask; its tiles are the
// global tiles [tileStart, tileStart + ceil(bytes / tile)).
constexpr int kMaxCopyTasks = 64;
struct CopyTask {
  const void* src;
  unsigned long long bytes, tileStart, dstOff, skipMask;
  int dstBase, ndst;
};
struct CopyArgs {
  CopyTask tasks[kMaxCopyTasks];
  void* dsts[kMaxCopyTasks];
  unsigned long long ntiles;       // tiles of all tasks
  unsigned long long timeoutNs;    // deadline of every wait for a bulk copy
  int* errClaim;
  ErrWord* err;
  int ntasks, tile, stages, pad;
};

// ---- direct collectives of one class in one launch: op i owns units
// [unitStart[i], unitStart[i + 1]) of the concatenated unit space (its
// `units` real ones, at least one so that some CTA owns its tail); pointers
// ptrs[ptrBase .. + nranks) send, then recv.
struct DirectOpDesc {
  unsigned long long count, chunk, inplaceMask, units;
  int coll, nranks, nsub, root, dtype, redop, vec, ptrBase;
  int postDiv, pad;
};
struct DirectBatchArgs {
  int nops, pad;
  unsigned long long unitStart[kMaxBatchOps + 1];
  DirectOpDesc ops[kMaxBatchOps];
  const void* ptrs[kMaxBatchPtrs];
};

// ---- channel partition (Sec. V-C): 16-byte packs spread over `nch` ranges,
// the first (packs % nch) ranges one pack longer, the element tail on the last.
VC_HD void channelRange(unsigned long long n, int unitBytes, int nch, int ch,
                        unsigned long long* start, unsigned long long* len) {
  unsigned long long epp = 16ull / (unsigned long long)unitBytes;
  unsigned long long npk = n / epp, tail = n % epp;
  unsigned long long base = npk / (unsigned long long)nch, rem = npk % (unsigned long long)nch;
  unsigned long long c = (unsigned long long)ch;
  unsigned long long sp = c * base + (c < rem ? c : rem);
  unsigned long long lp = base + (c < rem ? 1ull : 0ull);
  *start = sp * epp;
  *len = lp * epp + (ch == nch - 1 ? tail : 0ull);
}

// segment length of a ring-AllReduce loop at `off` in a channel ending at
// `end`: full loops use chunkCount; the last loop spreads the remainder over
// the k segments, rounded up to a pack
VC_HD unsigned long long ringLoopChunk(unsigned long long off, unsigned long long end, int k,
                                       unsigned long long chunk, int unitBytes) {
  unsigned long long epp = 16ull / (unsigned long long)unitBytes;
  unsigned long long loop = (unsigned long long)k * chunk;
  unsigned long long rem = end - off;
  if (rem >= loop) return chunk;
  unsigned long long c = (rem + (unsigned long long)k - 1) / (unsigned long long)k;
  return (c + epp - 1) / epp * epp;
}

VC_HD int modk(int a, int k) { return ((a % k) + k) % k; }

// ---- double binary tree (Sec. II-C).  Tree A: node i = rank + 1; odd nodes
// are leaves; an even node i with lowest set bit b has children i - b/2 and
// the first of i + b/2, i + b/4, ..., i + 1 not above k; the root is the
// largest power of two <= k.  Tree B mirrors A (k even) or shifts it by one
// rank (k odd).
VC_HD void treeANodeChildren(int k, int i, int* c0, int* c1) {
  *c0 = 0;
  *c1 = 0;
  if (i & 1) return;
  int b = i & -i;
  *c0 = i - b / 2;
  for (int d = b / 2; d >= 1; d >>= 1) {
    if (i + d <= k) { *c1 = i + d; break; }
  }
}
VC_HD int treeANodeParent(int k, int i) {
  int root = 1;
  while (root * 2 <= k) root *= 2;
  if (i == root) return 0;
  // walk down from the root: the parent is the node whose child is i
  int cur = root;
  while (true) {
    int c0, c1;
    treeANodeChildren(k, cur, &c0, &c1);
    if (c0 == i || c1 == i) return cur;
    // descend towards i: left subtree of cur holds nodes below cur
    cur = (i < cur) ? c0 : c1;
    if (cur == 0) return 0;   // not reachable (cannot happen for 1 <= i <= k)
  }
}
VC_HD int treeNodeOfRank(int k, int t, int r) {
  if (t == 0) return r + 1;
  if ((k & 1) == 0) return (k - 1 - r) + 1;
  return ((r + 1) % k) + 1;
}
VC_HD int treeRankOfNode(int k, int t, int i) {
  int ra = i - 1;
  if (t == 0) return ra;
  if ((k & 1) == 0) return k - 1 - ra;
  return ((ra - 1) % k + k) % k;
}
// parent rank (-1 at the root) and children ranks (-1 if absent), children in
// ascending tree-A node order
VC_HD void treeLinks(int k, int t, int r, int* parent, int* child0, int* child1) {
  int i = treeNodeOfRank(k, t, r);
  int c0, c1;
  treeANodeChildren(k, i, &c0, &c1);
  *child0 = c0 ? treeRankOfNode(k, t, c0) : -1;
  *child1 = c1 ? treeRankOfNode(k, t, c1) : -1;
  int p = treeANodeParent(k, i);
  *parent = p ? treeRankOfNode(k, t, p) : -1;
}

// ---- hierarchical tree (Sec. V-E: branching only across nodes, a chain
// inside each node).  The k vranks form k/m nodes of m consecutive vranks;
// the double binary tree above links the nodes; inside node n the chain runs
// n*m -> ... -> n*m+m-1 downwards, the node's first vrank hanging from the
// last vrank of its parent node and the node's last vrank carrying the first
// vranks of its child nodes, so no vrank has more than two children.
// m <= 1 is the flat tree.
VC_HD void treeLinksM(int k, int m, int t, int r, int* parent, int* child0, int* child1) {
  if (m <= 1) { treeLinks(k, t, r, parent, child0, child1); return; }
  const int nn = k / m, node = r / m, i = r % m;
  int pn = -1, c0 = -1, c1 = -1;
  if (nn > 1) treeLinks(nn, t, node, &pn, &c0, &c1);
  *parent = (i > 0) ? r - 1 : (pn >= 0 ? pn * m + m - 1 : -1);
  if (i < m - 1) {
    *child0 = r + 1;
    *child1 = -1;
  } else {
    *child0 = c0 >= 0 ? c0 * m : -1;
    *child1 = c1 >= 0 ? c1 * m : -1;
  }
}

}  // namespace vc
