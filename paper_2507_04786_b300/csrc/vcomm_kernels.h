// vcomm_kernels.h -- host-visible handles of the kernels in vcomm_kernels.cu.
#pragma once

namespace vc {
// persistent collective kernel for (protocol, dtype, op): AllReduce (ring and
// tree), ReduceScatter, Reduce and the single-rank copy
const void* reduceKernel(int proto, int dtype, int op);
// persistent byte-moving kernel for AllGather, Broadcast and the single-rank copy
const void* copyKernel(int proto);
// the serving layer's capped launch (vcomm_host.cu)
vResult_t serveCollective(int coll, const void* const* sendbufs, void* const* recvbufs, size_t count,
                          int dtype, int op, int proto, void* stream, vcomm_t c, int maxCtas,
                          vPlan_t* plan);

// direct protocol (vcomm_direct.cu): AllReduce / ReduceScatter / Reduce per
// (dtype, op); one byte-copy kernel for AllGather and Broadcast
const void* directKernel(int coll, int dtype, int op);
int directThreads(int coll, int dtype);   // the block size the kernel is compiled for
// a group's direct calls of one (dtype, op) class (or its copies), DirectBatchArgs;
// launched with directThreads(coll, dtype) threads
const void* directBatchKernel(int coll, int dtype, int op);
// AllReduce, ReduceScatter and Reduce of 16-byte aligned buffers staged
// through shared memory by bulk copies (DirectArgs with stages, tileBytes,
// timeoutNs, errClaim, err); one
// CTA per SM of directStagedThreads() threads and
// directStagedSmem(nranks, stages, tileBytes) bytes of dynamic shared memory
const void* directStagedKernel(int dtype, int op);
int directStagedThreads();
int directStagedMaxStages();
size_t directStagedSmem(int nranks, int stages, unsigned tileBytes);
// the largest tile (a multiple of 128 bytes, at most 16 KiB) whose staged
// shared memory fits smemMax bytes
unsigned directStagedTile(int nranks, int stages, size_t smemMax);
// copies staged through shared memory (CopyArgs); 32 threads per CTA,
// stages x tile + 8 x stages bytes of dynamic shared memory
const void* copyStagedKernel();
int copyStagedMaxStages();
// cluster protocol (vcomm_cluster_inst.cu): one cluster of nranks CTAs per channel
const void* clusterKernel(int dtype, int op);
const void* clusterCopyKernel();
constexpr int kClusterSmemBytes = 3 * 4 * 8192 + 256;   // == kCSmemBytes
constexpr int kClusterSlotBytes = 8192;                 // == kCSlotBytes
constexpr int kClusterSlots = 4;                        // == kCSlots
const void* debugEncodeKernel();
const void* debugDecodeKernel();
}  // namespace vc

namespace vc {
// the batched-launch kernel (vcomm_batch.cu); its parameter is a BatchArgs
const void* batchKernel();
// the persistent serving kernel (vcomm_batch.cu); its parameter is a ServeArgs
const void* serveKernel();
// serving mode 3 (vcomm_serve_tiles.cu): the resident tile kernel, a TileArgs;
// serveTilesThreads() threads per CTA and serveTilesSmem(stageBytes) bytes of
// dynamic shared memory (serveTilesStages() stages of stageBytes plus two
// output buffers of serveTilesOutBytes()); a register-path tile is a
// multiple of serveTilesUnitsPerIter() units
const void* serveTilesKernel();
// a group's direct calls as tiles of one launch (TileBatchArgs); same threads
// and shared memory as the serving tile kernel, one CTA per SM
const void* batchTilesKernel();
int serveTilesThreads();
int serveTilesUnitsPerIter();
int serveTilesStages();
unsigned serveTilesOutBytes();
size_t serveTilesSmem(unsigned stageBytes);
}  // namespace vc
