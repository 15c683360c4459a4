/*
 * vcomm.h -- C ABI of the virtual-rank collective library for sm_103a (B300).
 *
 * A communicator holds N virtual ranks ("vranks") on ONE GPU.  Each vrank has
 * its own caller-owned send and receive buffers in device memory; between two
 * vranks data moves only through per-connection FIFOs that the communicator
 * owns, in the same HBM.  With the paper's protocols (Simple, LL, LL128) a
 * collective runs as one persistent kernel per call: one CTA per (vrank,
 * channel) executes the paper's primitive step tables with flag-polled
 * synchronisation between CTAs.  Auto picks, on the ring, the direct protocol
 * (vProtoDirect below): a plain kernel with no FIFO and no flags that folds
 * each 16-byte unit's whole ring chain in the same order, so its results are
 * the Simple protocol's bit for bit.
 *
 * Paper: "Demystifying NCCL: An In-depth Analysis of GPU Communication
 * Protocols and Algorithms" (arXiv 2507.04786).  Section / table cited per call.
 *
 * Conventions shared by every call
 *  - sendbufs / recvbufs are HOST arrays of nranks DEVICE pointers, owned by the
 *    caller; the library copies the pointer arrays during the call and keeps no
 *    reference after it returns.  Each pointer must be aligned to the element
 *    size; 16-byte alignment (torch allocations) enables the vector path.
 *  - Calls are asynchronous: they return after enqueueing one kernel on
 *    `stream`; results are valid once the stream has been synchronised.
 *  - Synchronous errors (bad arguments, unsupported combinations, too many
 *    CTAs to be co-resident) are returned at once and nothing is enqueued.
 *  - Device-side failures (a flag wait that exceeded the deadline, an abort)
 *    end the kernel early; they are reported by vcommGetAsyncError.  The
 *    kernels never trap.  After such a failure the communicator returns the
 *    error from every later call until it is reset (vcommReset, which makes it
 *    usable again) or destroyed; vcommAbortPending ends in-flight calls first.
 *  - count == 0 is a successful no-op.
 *  - Calls on one communicator must be serialised on one stream (like NCCL
 *    calls on one communicator); calls on different communicators may overlap.
 */
#ifndef VCOMM_H_
#define VCOMM_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct vcomm* vcomm_t;
typedef void* vStream_t; /* a cudaStream_t; NULL is the legacy default stream */

typedef enum {
  vSuccess = 0,
  vInvalidArgument = 1,
  vUnsupported = 2,
  vOutOfMemory = 3,
  vCudaError = 4,
  vTimeout = 5,
  vAborted = 6,
  vInternalError = 7
} vResult_t;

/* Element types.  The paper names only the element notion (Sec. V-C: the
 * user type for reductions, bytes for AllGather / Broadcast); the list is
 * NCCL's.  Integers wrap (two's complement); floats round to nearest even
 * on every hop; 16-bit floats widen to fp32, combine and round once. */
typedef enum {
  vInt32 = 0, vFloat32 = 1, vFloat16 = 2, vBfloat16 = 3,
  vInt8 = 4, vUint8 = 5, vUint32 = 6, vInt64 = 7, vUint64 = 8, vFloat64 = 9
} vDataType_t;
/* Reductions f(received, local), each hop rounded to the element type.  max
 * and min keep the received operand on ties.  avg adds on every hop and
 * divides the completed value by nranks once, in the step that completes it
 * (the ring segment owner's recvReduceCopySend, the tree root, the
 * ReduceScatter / Reduce final recvReduceCopy): integers truncate toward
 * zero, floats round once.  The serving API and vAllReduceNoAlloc take
 * vSum / vMax on the first four types only. */
typedef enum { vSum = 0, vMax = 1, vProd = 2, vMin = 3, vAvg = 4 } vRedOp_t;
typedef enum { vAlgoAuto = 0, vAlgoRing = 1, vAlgoTree = 2 } vAlgo_t;
/* vProtoCluster has no counterpart in the paper: the LL line format of
 * Sec. III-B (4 data bytes + a 4-byte flag per 8-byte store) carried in
 * distributed shared memory instead of global memory.  Each channel's vranks
 * run as one thread-block cluster (CTA r = vrank r) and every FIFO lives in
 * its receiver's shared memory: 4 slots of 8 KiB (4 KiB of data) per
 * connection.  It needs nranks <= 16 (the largest cluster); Auto picks it for
 * tree AllReduce up to 256 KiB per rank on 2..16 vranks, where it is the
 * fastest FIFO protocol; a group of several calls and the serving API run it
 * as LL. */
/* vProtoDirect follows Sec. IV's P2P_DIRECT (ranks of one process move data
 * between source and destination buffers directly, with no intermediate
 * FIFO) to its end on one GPU: a thread reads the k input buffers of a
 * 16-byte unit and folds them in the ring schedule's order, so a call reads
 * each input byte once and writes each output byte once.  Ring algorithm
 * only; for a given plan (channels, chunkSteps) the results are the Simple
 * protocol's, bit for bit.  Auto picks it on the ring for nranks >= 2; a
 * group runs all its direct calls in one launch; the serving API runs it as
 * Simple.  An AllReduce on 2..16 vranks (fp64: up to 8), or a ReduceScatter
 * or Reduce on 2..4 vranks, of 16-byte aligned buffers of at least 8 MiB per
 * rank (send buffer; env VCOMM_STAGED_MIN_BYTES, read at vcommInit) moves its
 * data by bulk
 * asynchronous copies through shared memory (same fold, same bits); so do an AllGather or Broadcast of 16-byte aligned
 * buffers whose per-rank size is whole 16-byte units and at least that
 * threshold.  A bulk copy that does not complete within timeoutSec fails the
 * call with vTimeout like a flag wait. */
typedef enum {
  vProtoAuto = 0,
  vProtoSimple = 1,
  vProtoLL = 2,
  vProtoLL128 = 3,
  vProtoCluster = 4,
  vProtoDirect = 5
} vProto_t;

#define VCOMM_MAX_RANKS 64
#define VCOMM_MAX_CHANNELS 64

/* Communicator configuration.  Zero fields take the defaults in brackets,
 * which follow the paper's Table "NCCL channel buffer sizes" (Sec. V-C). */
typedef struct {
  size_t slotBytes[3];   /* FIFO slot bytes for Simple, LL, LL128 [512 KiB, 32 KiB, 600 KiB] */
  int nsteps;            /* slots per connection FIFO, NCCL_STEPS of Sec. V-C [8] */
  int nthreads;          /* upper bound on threads per CTA [1024; Simple kernels use at most
                            512]; lowered to fit co-residency */
  double timeoutSec;     /* deadline of every device flag wait [5 s; env VCOMM_TIMEOUT_MS] */
  int treeNodeSize;      /* vranks per node of the tree algorithm [1]: the double binary tree
                            branches only across nodes of this many consecutive vranks, which
                            form a chain inside the node (Sec. V-E); must divide nranks */
} vcommConfig_t;

/* Plan of one call: algorithm, protocol, channels and chunk steps.  Used to
 * pin a plan (vcommSetPlan) and to read back the plan of the last call. */
typedef struct {
  vAlgo_t algo;
  vProto_t proto;
  int nchannels;         /* channels (CTAs per vrank; Tree uses two per channel) */
  int chunkSteps;        /* FIFO slots per chunk: chunkCount = slot data * chunkSteps */
} vPlan_t;

/* ncclCommInitAll (Sec. II-A-1): one communicator over `nranks` vranks with
 * up to `nchannels` channels (Sec. II-C).  nranks in [1, 64], nchannels in
 * [1, 64].  Uses the current CUDA device.  FIFO arenas are allocated lazily
 * per (algorithm, protocol) on first use, or eagerly by vcommPrepare.
 * Errors: vInvalidArgument (ranges, NULL), vOutOfMemory, vCudaError. */
vResult_t vcommInit(vcomm_t* comm, int nranks, int nchannels);
vResult_t vcommInitConfig(vcomm_t* comm, int nranks, int nchannels, const vcommConfig_t* cfg);

/* Allocate the FIFO arenas for the given algorithms and protocols now
 * (bit i of algoMask = vAlgo_t i, bit i of protoMask = vProto_t i), so that
 * later calls allocate nothing (e.g. before CUDA-graph capture). */
vResult_t vcommPrepare(vcomm_t comm, unsigned algoMask, unsigned protoMask);

/* ncclCommDestroy (Sec. II-A-1): waits for all work on the device, then frees
 * the FIFO arenas and the communicator.  NULL is a no-op. */
vResult_t vcommDestroy(vcomm_t comm);

/* ncclCommAbort (Sec. II-A-1): raises the abort word that every device flag
 * wait polls, so in-flight kernels of this communicator return early, then
 * waits for the device and frees the communicator. */
vResult_t vcommAbort(vcomm_t comm);

/* Recovery (Sec. II-A-1: abort is "intended for error recovery").
 * vcommAbortPending raises the abort word like vcommAbort, waits until the
 * in-flight kernels have returned (their waits end with vAborted), and keeps
 * the communicator.  vcommReset makes a failed or aborted communicator usable
 * again: it waits for the device, re-zeroes every FIFO arena and its
 * counters (a failed call leaves them half written), clears the error and
 * abort words and the debug fault injection.  It must not be called with
 * work of this communicator still to be launched (inside a group: error). */
vResult_t vcommAbortPending(vcomm_t comm);
vResult_t vcommReset(vcomm_t comm);

/* Asynchronous error of the communicator: vSuccess, vTimeout (a flag wait hit
 * its deadline) or vAborted.  Does not synchronise. */
vResult_t vcommGetAsyncError(vcomm_t comm, vResult_t* err);

/* Pin the plan used by later calls whose algo/proto arguments are Auto and
 * set their channels / chunk steps (fields equal to 0 or Auto stay with the
 * tuner).  NULL clears the pin. */
vResult_t vcommSetPlan(vcomm_t comm, const vPlan_t* plan);

/* The plan the last call on this communicator ran with. */
vResult_t vcommGetLastPlan(vcomm_t comm, vPlan_t* plan);

/* ncclAllReduce (Sec. II-A-2).  Ring: Sec. V-E, Table "Ring AllReduce";
 * Tree: double binary tree, Sec. II-C and Table "Tree AllReduce".
 * recvbufs[r] = op over j of sendbufs[j], `count` elements each, for every r.
 * In place when sendbufs[r] == recvbufs[r]. */
vResult_t vAllReduce(const void* const* sendbufs, void* const* recvbufs, size_t count,
                     vDataType_t dtype, vRedOp_t op, vAlgo_t algo, vProto_t proto,
                     vStream_t stream, vcomm_t comm);

/* ncclReduceScatter (Sec. II-A-2), ring only (Table "Ring ReduceScatter").
 * sendbufs[r] holds nranks blocks of recvcount elements; recvbufs[r] receives
 * the reduction of block r.  In place when recvbufs[r] == sendbufs[r] +
 * r * recvcount elements. */
vResult_t vReduceScatter(const void* const* sendbufs, void* const* recvbufs, size_t recvcount,
                         vDataType_t dtype, vRedOp_t op, vAlgo_t algo, vProto_t proto,
                         vStream_t stream, vcomm_t comm);

/* ncclAllGather (Sec. II-A-2), ring only (Table "Ring AllGather").
 * recvbufs[r] holds nranks blocks of sendcount elements; block b is rank b's
 * sendbuf.  Data moves as bytes (Sec. V-C).  In place when sendbufs[r] ==
 * recvbufs[r] + r * sendcount elements. */
vResult_t vAllGather(const void* const* sendbufs, void* const* recvbufs, size_t sendcount,
                     vDataType_t dtype, vAlgo_t algo, vProto_t proto, vStream_t stream,
                     vcomm_t comm);

/* ncclBroadcast (Sec. II-A-2), ring chain from `root` (Table "Ring
 * Broadcast").  recvbufs[r] = sendbufs[root] for all r; only sendbufs[root]
 * is read (others may be NULL).  ncclBcast's in-place form is
 * sendbufs[root] == recvbufs[root]. */
vResult_t vBroadcast(const void* const* sendbufs, void* const* recvbufs, size_t count,
                     vDataType_t dtype, int root, vAlgo_t algo, vProto_t proto,
                     vStream_t stream, vcomm_t comm);

/* ncclReduce (Sec. II-A-2), ring chain ending at `root` (Table "Ring
 * Reduce").  Only recvbufs[root] is written (others may be NULL). */
vResult_t vReduce(const void* const* sendbufs, void* const* recvbufs, size_t count,
                  vDataType_t dtype, vRedOp_t op, int root, vAlgo_t algo, vProto_t proto,
                  vStream_t stream, vcomm_t comm);

/* ---- group calls: many collectives, one launch ---------------------------
 * ncclGroupStart / ncclGroupEnd (Sec. II-A-4).  Collective calls between
 * vGroupStart and vGroupEnd (on the calling host thread; groups nest) are
 * validated and planned immediately but not launched; vGroupEnd launches, per
 * communicator, at most two persistent kernels.  The FIFO-protocol calls run
 * in ONE batch kernel: up to 4 gangs of (nranks x nch/G) CTAs run their share
 * of the calls (longest first) concurrently, each gang's calls one after
 * another through the same FIFOs.  The direct-protocol calls (Auto's choice
 * on the ring) run in ONE launch of the tile engine on up to 16 vranks with
 * sum / max of 32- and 16-bit types (any other direct group: one launch per
 * (dtype, op) class, and one for the copies): every call is cut into tiles,
 * laid end to end and shared out statically, one CTA per SM; a tile of
 * 16-byte aligned buffers moves through shared memory by bulk copies (a
 * producer warp issues them while eight consumer warps fold), other tiles
 * take element-wise loads and stores.  Env VCOMM_TILE_GROUPS=0 (read at
 * vcommInit) keeps the per-class launches.  Each call's result is
 * bit-identical to the same call launched alone with the plan
 * vcommGetGroupPlans reports.  All
 * calls of one communicator in a group must use the same stream.  The launch
 * is capturable in a CUDA graph once the arenas it needs exist (vcommPrepare,
 * or one uncaptured run); the batch description is a kernel parameter, so a
 * replay needs no host memory.  Calls within a group return vSuccess after
 * validation; vGroupEnd returns the first launch error.  The buffers of
 * every call must stay allocated until the group's work has completed on
 * the stream (nothing is read before vGroupEnd). */
vResult_t vGroupStart(void);
vResult_t vGroupEnd(void);

/* Plans of the calls of the last group launched on `comm`, in call order
 * (channels may be lower than requested: a gang has nch/G channels).
 * Point-to-point transfers have no plan and are not listed. */
vResult_t vcommGetGroupPlans(vcomm_t comm, vPlan_t* plans, int maxPlans, int* nPlans);

/* ---- point-to-point (Sec. II-A-3: ncclSend / ncclRecv) --------------------
 * vSend: vrank `rank` sends `count` elements from `sendbuf` (device) to vrank
 * `peer`; vRecv: vrank `rank` receives `count` elements from vrank `peer`
 * into `recvbuf` (device).  Every vrank lives in this process, so both sides
 * of a transfer must be issued inside one vGroupStart / vGroupEnd; there the
 * i-th send from a to b meets the i-th receive at b from a, and their counts
 * and dtypes must agree (else vGroupEnd returns vInvalidArgument and runs
 * nothing of the group).  rank == peer is a local copy.  Same-process ranks
 * copy directly from the source to the destination buffer (Sec. IV,
 * P2P_DIRECT); each transfer is its own task of one launch, so grouped
 * transfers run concurrently (Sec. II-C).  When every transfer of the group
 * is 16-byte aligned and whole 16-byte units and the group moves at least
 * VCOMM_STAGED_MIN_BYTES (8 MiB), the tasks move by bulk copies through
 * shared memory, up to 64 per launch.  Buffers are caller-owned and must
 * be element-aligned; a receive buffer must not overlap another transfer's
 * buffers.  Calls outside a group return vInvalidArgument. */
vResult_t vSend(const void* sendbuf, size_t count, vDataType_t dtype, int rank, int peer,
                vcomm_t comm, vStream_t stream);
vResult_t vRecv(void* recvbuf, size_t count, vDataType_t dtype, int rank, int peer,
                vcomm_t comm, vStream_t stream);

/* All-to-all as the grouped send / receive pattern of Sec. II-A-4: block j
 * (`count` elements) of sendbufs[r] lands in block r of recvbufs[j], for all
 * r, j.  Both arrays hold nranks device pointers of nranks x count elements.
 * Inside a group it adds its nranks^2 transfers to the group; outside, it
 * launches them at once.  A receive buffer may not overlap any send or other
 * receive buffer (no in-place form, except on one vrank). */
vResult_t vAllToAll(const void* const* sendbufs, void* const* recvbufs, size_t count,
                    vDataType_t dtype, vcomm_t comm, vStream_t stream);

/* ---- autotuner ------------------------------------------------------------
 * Protocol / algorithm / channel selection (Sec. III-D; Sec. II-C: "the tuning
 * model determines how many channels"): times every candidate plan
 * (ring/tree x Simple/LL/LL128 x channels 1, 2, 4, ... nch, plus the cluster
 * protocol up to 4 MiB on <= 16 vranks and the direct protocol on the ring)
 * on this device at
 * per-rank sizes 1 KiB x 4^i <= maxBytes for each collective whose bit is set
 * in collMask (bit 0 AllReduce, 1 ReduceScatter, 2 AllGather, 3 Broadcast,
 * 4 Reduce) and keeps the fastest per size.  Later calls with Auto arguments
 * take their plan from the table at the nearest size (log scale).  Allocates
 * 2 x nranks x maxBytes of scratch for the duration of the call; synchronous. */
vResult_t vcommTune(vcomm_t comm, unsigned collMask, size_t maxBytes, vStream_t stream);

/* The tuned table of one collective (0..4 as in collMask): per size bucket the
 * chosen plan, the per-rank size in bytes and the measured time in us. */
vResult_t vcommGetTuneTable(vcomm_t comm, int coll, vPlan_t* plans, size_t* bytes, float* usec,
                            int maxEntries, int* nEntries);

/* ---- serving: continuous batching of collective requests ------------------
 * No counterpart in the paper beyond its collectives.  A server runs one
 * persistent kernel whose gangs each execute one request at a time: one wide
 * gang (bigGangChannels x maxRanks CTAs) for requests whose per-rank size is
 * >= bigThreshold, and smallGangs narrow gangs (maxRanks CTAs) for the rest;
 * a request of k vranks spreads over its gang as (gang CTAs / k) channels.  A host thread admits submitted requests in arrival order --
 * a request that must wait does not block later ones -- as soon as the bytes
 * of all admitted, unreleased requests (send + receive, all vranks) fit in
 * memBudget and a suitable gang is free; it allocates the request's receive
 * buffers from a pool of memBudget bytes, posts the request to the gang's
 * host-mapped mailbox, and records its completion time.  A request's plan
 * depends only on the request (protocol by size unless given; one channel,
 * or all of the wide gang's channels for large requests; chunkSteps 1), so
 * its result is bit-identical alone and in any mix, and equal to vAllReduce
 * (ring) with that plan.  mode 1 ("plain") runs the same requests as one
 * ordinary launch each on one stream, for comparison.  mode 2 ("streams")
 * is continuous batching without a resident kernel: each admitted request is
 * one launch on a lane -- a stream for large requests (>= bigThreshold) and
 * max(1, smallGangs) streams for the others -- whose grid is capped (the
 * large lane leaves 16 SMs; a small lane takes one CTA per 256 KiB of the
 * request's traffic, 4 to 32), so that requests on different lanes run side
 * by side; at most two launches per lane are in flight.  With the paper's
 * FIFO protocols, requests of the same vrank count share one communicator's
 * FIFO arena, so each such launch waits on the device for the previous one
 * (whatever its lane); direct-protocol requests have no FIFO and overlap
 * freely.  Plans as in mode 1, so results are bit-identical across modes.
 * mode 3 ("tiles") is continuous batching for the direct protocol (Auto):
 * one resident kernel; its CTA 0 takes requests in arrival order from a ring
 * in host-mapped memory and queues them on the device, small requests
 * (< bigThreshold per rank) ahead of large ones, and every other CTA takes
 * the next tile (a byte range of one block, at most ~4 MiB of traffic) of the
 * first queued request that has tiles left; the tiles of 16-byte aligned
 * buffers move through shared memory by bulk copies (the group launch's
 * tile engine).  So a request starts as soon as a CTA is free, small
 * requests overtake large ones at tile boundaries (unless the first large
 * request was queued 0.5 ms before the first small one), and the CTA that finishes
 * a request's last tile reports its completion to host memory.  Plans as in mode 1 (results bit-identical); other protocols are
 * refused (vUnsupported).  The kernel returns after idleTimeoutSec without
 * work and is started again by the next request.
 * While a mode-0 or mode-3 server exists its kernel occupies the SMs: do not
 * launch and wait for other kernels meanwhile (copies are fine). */
typedef enum { vCollAllReduce = 0, vCollReduceScatter = 1, vCollAllGather = 2 } vColl_t;
typedef struct vserve* vserve_t;
typedef struct {
  int mode;              /* 0 continuous batching on resident gangs [default], 1 one launch
                            per request, 2 continuous batching on lanes of streams, 3
                            continuous batching of direct-protocol tiles */
  int maxRanks;          /* vranks per request, <= 16 [16] */
  size_t memBudget;      /* bytes of request buffers in flight [40 GiB]; the pool is this size */
  int bigGangChannels;   /* channels of the wide gang [0: every co-resident CTA the
                            narrow gangs leave, 8 on a B300 at 512 threads] */
  int smallGangs;        /* narrow gangs [1] */
  size_t bigThreshold;   /* per-rank bytes from which a request is large [4 MiB] */
  size_t slotBytes[3];   /* FIFO slots, Simple / LL / LL128 [256 KiB, 32 KiB, 300 KiB] */
  double idleTimeoutSec; /* the kernel stops after this long without a request [30 s] */
  int threads;           /* threads per CTA of the serving kernel, <= 512 [512] */
} vserveConfig_t;
typedef struct {
  uint64_t submitted, completed, failed, queued;
  size_t inflightBytes, maxInflightBytes;
} vserveStats_t;

vResult_t vServeCreate(vserve_t* server, const vserveConfig_t* cfg);
/* Queue one request: sendbufs = nranks device pointers (caller-owned, must stay
 * valid until completion), count as in the collective (AllReduce count,
 * ReduceScatter recvcount, AllGather sendcount).  flags bit 0: release the
 * receive buffers at completion (results are not kept).  arrivalNs: the
 * request's arrival on the CLOCK_MONOTONIC clock (0: now), the origin of its
 * latency.  Returns a ticket. */
vResult_t vServeSubmit(vserve_t server, int coll, const void* const* sendbufs, size_t count,
                       vDataType_t dtype, vRedOp_t op, int nranks, vProto_t proto, int flags,
                       int64_t arrivalNs, uint64_t* ticket);
/* state: 0 queued, 1 running, 2 done, 3 failed; latency = completion - arrival
 * (ns, -1 until done); service = the request's own run time on the device
 * (mode 0: the gang's clock; modes 1, 2: events around its launch; ns); plan; recvbufs (nranks pointers into the
 * pool, valid until vServeRelease).  Any output may be NULL except state. */
vResult_t vServeQuery(vserve_t server, uint64_t ticket, int* state, int64_t* latencyNs,
                      int64_t* serviceNs, vPlan_t* plan, void** recvbufs);
/* Forget a finished request and return its buffers to the budget. */
vResult_t vServeRelease(vserve_t server, uint64_t ticket);
vResult_t vServeGetStats(vserve_t server, vserveStats_t* stats);
/* Stops the kernel after the running requests, then frees everything. */
vResult_t vServeDestroy(vserve_t server);

/* ---- allocation-free AllReduce -----------------------------------------
 * The paper has no counterpart to this entry point.  It exists for callers
 * that cannot call cudaMalloc at the point where they need an AllReduce: code
 * that must stay inside a fixed memory budget owned by another allocator, and
 * latency-critical code where cudaMalloc / cudaFree could block or
 * synchronise the device.  It runs the ring AllReduce with the Simple protocol
 * (same kernel and same results as vAllReduce with algo Ring, proto Simple,
 * nchannels channels, 64 KiB Simple slots and chunkSteps 1), but its FIFOs,
 * counters and error words live in one fixed device array that the library
 * defines at file scope: VCOMM_NOALLOC_SCRATCH_BYTES (about 8 MiB) on every
 * GPU that loads the library, held until the process exits.  No
 * communicator is needed and nothing is allocated.
 *  - nranks x nchannels must not exceed VCOMM_NOALLOC_MAX_CONNS (32): larger
 *    requests return vInvalidArgument and enqueue nothing.  count is not
 *    limited (data streams through the FIFOs).
 *  - The first call on a device looks up the array's device address (with
 *    that device current); make that first call before any stream capture.
 *    The address is kept for the life of the process, so calls must not span
 *    a cudaDeviceReset of the device.  Device ordinals up to 63.
 *  - Every call shares the one array and clears its counters first, so calls
 *    that overlap on the GPU (other streams, other host threads) race and
 *    corrupt each other: serialise them.
 *  - deviceStatus: NULL, or caller-owned device memory of 4 ints that the call
 *    sets to {code, rank, channel, where} of a device-side failure (a flag wait
 *    past its 5 s deadline), or to zeros on success.  With NULL a device-side
 *    failure is recorded only inside the library's array, where the caller
 *    cannot read it: pass a status buffer to observe timeouts.
 * Other arguments and in-place rules as in vAllReduce. */
#define VCOMM_NOALLOC_MAX_CONNS 32
#define VCOMM_NOALLOC_SCRATCH_BYTES 8398080
vResult_t vAllReduceNoAlloc(const void* const* sendbufs, void* const* recvbufs, size_t count,
                            vDataType_t dtype, vRedOp_t op, int nranks, int nchannels,
                            int* deviceStatus, vStream_t stream);

/* Library version, e.g. 100 for 0.1.0. */
int vcommVersion(void);

/* ---- protocol encoders exposed for testing (Sec. III-B, III-C) ----------
 * Run the device-side LL / LL128 line encoder on `nbytes` bytes at device
 * pointer `src` with the given flag and write the lines to device pointer
 * `lines` (LL: 8 bytes per 4 data bytes, rounded up to an even number of
 * lines; LL128: 128 bytes per 120 data bytes).  Decoding runs the device
 * reader, which fails with vTimeout if a line never carries `flag`. */
vResult_t vDebugEncode(vProto_t proto, const void* src, size_t nbytes, uint64_t flag,
                       void* lines, vStream_t stream);
vResult_t vDebugDecode(vProto_t proto, const void* lines, size_t nbytes, uint64_t flag,
                       void* dst, double timeoutSec, vStream_t stream);

/* Per-hop latency of the FIFO protocols (Sec. III quotes ~6 / ~1 / ~2 us per
 * hop for Simple / LL / LL128): a ring of n CTAs (one warp each) passes one
 * FIFO line around `laps` times -- LL: one 8-byte {data, flag} line; LL128:
 * one 128-byte line written by 8 lanes, the flag in its last 8 bytes;
 * Simple: a 128-byte payload, a fence and a release store of a counter that
 * the receiver acquires -- and *nsPerHop = elapsed %globaltimer / (laps x n).
 * ringSms: n SM ids (%smid, distinct, < 1024), position i of the ring on SM
 * ringSms[i] (the kernel runs one CTA on every SM; n <= SM count); NULL: the
 * ring is one thread-block cluster of n <= 16 CTAs (one GPC).  smOut (may be
 * NULL): n ints, the SM id of each position.  Every wait is bounded by
 * timeoutSec (vTimeout, e.g. for an SM id no SM has).  Allocates a few KB,
 * synchronous; vInvalidArgument for n < 2, laps < 1, bad ids or protocols. */
/* The tiles the tile engine (group calls, serving mode 3; no paper
 * counterpart) cuts a direct-protocol op into: host arithmetic only, no
 * device needed.  coll: 0 AllReduce, 1 ReduceScatter, 2 AllGather,
 * 3 Broadcast, 4 Reduce; count in elements (AllReduce, ReduceScatter's
 * recvcount, Reduce) or bytes (AllGather's sendcount, Broadcast);
 * dtypeSize 1, 2 or 4; vec as the direct protocol's access kind (0 element
 * accesses, 1 aligned 16-byte units, 2 aligned buffers whose RS / AG blocks
 * are not whole units); workers: the CTAs that take tiles; iter: units per
 * register-path iteration; shared: 1 for a group launch (tiles shared out
 * statically), 0 for serving (claimed one at a time).  out[8]: staged (1: byte ranges of a block moved
 * by bulk copies), units and tileUnits (register path), blockBytes,
 * tileBytes and perBlock (staged: bytes of a block moved by bulk copies, per
 * tile, tiles per block), ntiles, and the access kind the engine uses.
 * vInvalidArgument for out == NULL or arguments out of range. */
vResult_t vDebugTileGeometry(int coll, int nranks, unsigned long long count, int dtypeSize, int vec,
                             unsigned long long workers, unsigned long long iter, int shared,
                             unsigned long long* out);

vResult_t vDebugHopLatency(vProto_t proto, const int* ringSms, int n, int laps, double timeoutSec,
                           double* nsPerHop, int* smOut);

/* Fault injection for tests of failure detection: from the next call on,
 * vrank `rank`'s CTAs return without taking part (-1 turns it off), so the
 * other vranks' flag waits run into their deadline (vTimeout) or the abort
 * word (vAborted) -- a lost peer, simulated without any GPU fault. */
vResult_t vcommDebugSetSkipRank(vcomm_t comm, int rank);

#ifdef __cplusplus
}
#endif
#endif /* VCOMM_H_ */
