/*
 * vcomm_oracle.c -- plain, slow CPU model of the virtual-rank collectives.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * calls this file.  Only the tests, the smoke check and the CPU-baseline leg of
 * the benchmark use it.  It shares no code, header, table or constant with the
 * CUDA path: everything here is re-derived from the paper ("Demystifying NCCL",
 * arXiv 2507.04786) and from IEEE 754.
 *
 * What it models (paper section / table in brackets):
 *   - channel partition, outer loops and chunks          [Sec. V-C, Table "buffer sizes"]
 *   - ring AllReduce step table                          [Sec. V-E, Table "Ring AllReduce"]
 *   - ring ReduceScatter / AllGather step tables         [Sec. V-E, Tables "Ring RS", "Ring AG"]
 *   - ring Broadcast / Reduce chains                     [Sec. V-E, Tables "Ring Broadcast", "Ring Reduce"]
 *   - double-binary-tree AllReduce                       [Sec. II-C; Sec. V-E, Table "Tree AllReduce"]
 *   - LL (4 B data + 4 B flag) and LL128 (120 B + 8 B) line encodings [Sec. III-B, III-C]
 *
 * Readings taken where the paper is silent (each is listed in the design notes):
 *   R1 partition: 16-byte packs spread over channels, the first (packs % C)
 *      channels get one extra pack, the element tail goes to the last channel.
 *   R2 ring: at step t rank r works on segment (r - t - 1) mod k, so rank r
 *      completes segment r at step k-1.
 *   R3 every hop rounds to the user dtype (the FIFO holds the user dtype);
 *      the reduction is f(received, local); sum is IEEE round-to-nearest-even,
 *      max keeps the received operand on ties.
 *   R4 chain Reduce starts at the root's ring successor; Broadcast runs
 *      root, root+1, ..., root-1.
 *   R5 double binary tree: tree A over nodes i = r + 1, tree B by mirror (k
 *      even) or shift by one (k odd); the data of each channel is split into two
 *      halves, the first on tree A and the second on tree B.
 *   R18 ops and dtypes beyond the paper's examples: prod rounds each hop's
 *      product to the dtype like sum; min keeps the received operand on ties
 *      like max; integers (8, 32, 64 bits, signed or not) wrap; avg adds on
 *      every hop and divides the completed value by the number of ranks in
 *      the one step that completes it (recvReduceCopy / recvReduceCopySend:
 *      the ring segment owner, the tree root, the Reduce root), integers
 *      truncating toward zero, floats rounding once.
 *
 * Arithmetic: values are widened exactly to double, combined in double and
 * rounded once to the user dtype with the encoders below (own implementation
 * of IEEE 754 round-to-nearest-even).  For a single addition the double
 * intermediate is innocuous (53 >= 2p + 2 for p = 24, 11, 8), so every hop
 * yields the correctly rounded dtype sum.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

/* dtype codes (oracle-private) */
enum {
  O_INT32 = 0, O_FP32 = 1, O_FP16 = 2, O_BF16 = 3, O_BYTE = 4,
  O_INT8 = 5, O_UINT8 = 6, O_UINT32 = 7, O_INT64 = 8, O_UINT64 = 9, O_FP64 = 10
};
/* reduction codes.  avg is the sum whose final value is divided by the
 * number of ranks where the schedule completes it (reading R18). */
enum { O_SUM = 0, O_MAX = 1, O_PROD = 2, O_MIN = 3, O_AVG = 4 };
/* protocol codes */
enum { O_SIMPLE = 0, O_LL = 1, O_LL128 = 2 };
/* primitive codes, named after Sec. V-B */
enum {
  P_NONE = 0, P_SEND = 1, P_RECV = 2, P_RECV_REDUCE_SEND = 3, P_RECV_COPY_SEND = 4,
  P_RECV_REDUCE_COPY_SEND = 5, P_COPY_SEND = 6, P_RECV_REDUCE_COPY = 7
};

int o_dtype_size(int dt) {
  switch (dt) {
    case O_INT32: case O_FP32: case O_UINT32: return 4;
    case O_FP16: case O_BF16: return 2;
    case O_BYTE: case O_INT8: case O_UINT8: return 1;
    case O_INT64: case O_UINT64: case O_FP64: return 8;
  }
  return 0;
}

static int o_is_int(int dt) {
  return dt == O_INT32 || dt == O_INT8 || dt == O_UINT8 || dt == O_UINT32 || dt == O_INT64 ||
         dt == O_UINT64;
}
static int o_is_signed(int dt) { return dt == O_INT32 || dt == O_INT8 || dt == O_INT64; }

/* ------------------------------------------------------------------------ */
/* IEEE 754 binary formats: exact decode and round-to-nearest-even encode.   */
/* ------------------------------------------------------------------------ */

/* round a non-negative double that is an exact multiple of 1/2 ... to an
 * integer, ties to even.  y < 2^53 so floor and the difference are exact. */
static double o_round_half_even(double y) {
  double f = floor(y);
  double d = y - f;
  if (d > 0.5) return f + 1.0;
  if (d < 0.5) return f;
  return (fmod(f, 2.0) == 0.0) ? f : f + 1.0;
}

/* Encode x into a binary format with `ebits` exponent bits and `mbits`
 * fraction bits (bias 2^(ebits-1)-1), rounding to nearest, ties to even,
 * with gradual underflow and overflow to infinity. */
static uint32_t o_encode_float(double x, int ebits, int mbits) {
  const int bias = (1 << (ebits - 1)) - 1;
  const int emin = 1 - bias;              /* exponent of the smallest normal */
  const int emax = bias;                  /* exponent of the largest finite  */
  const uint32_t expmask = (1u << ebits) - 1u;
  uint32_t sign = signbit(x) ? 1u : 0u;
  uint32_t sbit = sign << (ebits + mbits);
  if (isnan(x)) return sbit | (expmask << mbits) | (1u << (mbits - 1));
  double ax = fabs(x);
  if (isinf(ax)) return sbit | (expmask << mbits);
  if (ax == 0.0) return sbit;
  int e2;
  (void)frexp(ax, &e2);                   /* ax = m * 2^e2, m in [0.5, 1) */
  int e = e2 - 1;                         /* ax in [2^e, 2^(e+1)) */
  if (e < emin) {
    /* subnormal: count units of 2^(emin - mbits) */
    double q = o_round_half_even(ldexp(ax, mbits - emin));
    /* q == 2^mbits becomes the smallest normal, which the bit pattern encodes naturally */
    return sbit | (uint32_t)q;
  }
  double q = o_round_half_even(ldexp(ax, mbits - e));   /* in [2^mbits, 2^(mbits+1)] */
  if (q == ldexp(1.0, mbits + 1)) { q = ldexp(1.0, mbits); e += 1; }
  if (e > emax) return sbit | (expmask << mbits);
  uint32_t frac = (uint32_t)(q - ldexp(1.0, mbits));
  return sbit | ((uint32_t)(e + bias) << mbits) | frac;
}

static double o_decode_float(uint32_t bits, int ebits, int mbits) {
  const int bias = (1 << (ebits - 1)) - 1;
  const uint32_t expmask = (1u << ebits) - 1u;
  uint32_t sign = (bits >> (ebits + mbits)) & 1u;
  uint32_t ex = (bits >> mbits) & expmask;
  uint32_t frac = bits & ((1u << mbits) - 1u);
  double v;
  if (ex == expmask) v = frac ? NAN : INFINITY;
  else if (ex == 0) v = ldexp((double)frac, 1 - bias - mbits);
  else v = ldexp((double)(frac | (1u << mbits)), (int)ex - bias - mbits);
  return sign ? -v : v;
}

uint16_t o_f64_to_f16(double x) { return (uint16_t)o_encode_float(x, 5, 10); }
uint16_t o_f64_to_bf16(double x) { return (uint16_t)o_encode_float(x, 8, 7); }
uint32_t o_f64_to_f32bits(double x) { return o_encode_float(x, 8, 23); }
double o_f16_to_f64(uint16_t b) { return o_decode_float(b, 5, 10); }
double o_bf16_to_f64(uint16_t b) { return o_decode_float(b, 8, 7); }
double o_f32bits_to_f64(uint32_t b) { return o_decode_float(b, 8, 23); }

/* bulk conversions used by the Python side to build fp16/bf16 inputs and
 * fp64 reference sums */
void o_encode_array(int dt, const double* x, size_t n, void* out) {
  for (size_t i = 0; i < n; i++) {
    switch (dt) {
      case O_FP16: ((uint16_t*)out)[i] = o_f64_to_f16(x[i]); break;
      case O_BF16: ((uint16_t*)out)[i] = o_f64_to_bf16(x[i]); break;
      case O_FP32: ((uint32_t*)out)[i] = o_f64_to_f32bits(x[i]); break;
      default: break;
    }
  }
}
void o_decode_array(int dt, const void* in, size_t n, double* x) {
  for (size_t i = 0; i < n; i++) {
    switch (dt) {
      case O_FP16: x[i] = o_f16_to_f64(((const uint16_t*)in)[i]); break;
      case O_BF16: x[i] = o_bf16_to_f64(((const uint16_t*)in)[i]); break;
      case O_FP32: x[i] = o_f32bits_to_f64(((const uint32_t*)in)[i]); break;
      case O_INT32: x[i] = (double)((const int32_t*)in)[i]; break;
      default: break;
    }
  }
}

/* ------------------------------------------------------------------------ */
/* One reduction: out = f(a, b) with a the received operand, b the local one */
/* [Sec. V-B: recvReduce* "receives ... performs an element-wise reduction   */
/*  with its local buffer"]; result rounded to the dtype (reading R3).      */
/* ------------------------------------------------------------------------ */
static double o_get(int dt, const void* p, size_t i) {
  switch (dt) {
    case O_FP64: { double v; memcpy(&v, (const char*)p + 8 * i, 8); return v; }
    case O_FP32: { uint32_t b; memcpy(&b, (const char*)p + 4 * i, 4); return o_f32bits_to_f64(b); }
    case O_FP16: return o_f16_to_f64(((const uint16_t*)p)[i]);
    case O_BF16: return o_bf16_to_f64(((const uint16_t*)p)[i]);
  }
  return 0.0;
}
static void o_put(int dt, void* p, size_t i, double v) {
  switch (dt) {
    case O_FP64: memcpy((char*)p + 8 * i, &v, 8); break;
    case O_FP32: { uint32_t b = o_f64_to_f32bits(v); memcpy((char*)p + 4 * i, &b, 4); break; }
    case O_FP16: ((uint16_t*)p)[i] = o_f64_to_f16(v); break;
    case O_BF16: ((uint16_t*)p)[i] = o_f64_to_bf16(v); break;
  }
}

/* integer element i as a 64-bit pattern: sign-extended for signed types,
 * zero-extended for unsigned ones */
static uint64_t o_geti(int dt, const void* p, size_t i) {
  switch (dt) {
    case O_INT8: return (uint64_t)(int64_t)((const int8_t*)p)[i];
    case O_UINT8: return (uint64_t)((const uint8_t*)p)[i];
    case O_INT32: return (uint64_t)(int64_t)((const int32_t*)p)[i];
    case O_UINT32: return (uint64_t)((const uint32_t*)p)[i];
    case O_INT64: case O_UINT64: { uint64_t v; memcpy(&v, (const char*)p + 8 * i, 8); return v; }
  }
  return 0;
}
/* store the low bits (two's-complement wraparound) */
static void o_puti(int dt, void* p, size_t i, uint64_t v) {
  switch (dt) {
    case O_INT8: case O_UINT8: ((uint8_t*)p)[i] = (uint8_t)v; break;
    case O_INT32: case O_UINT32: { uint32_t w = (uint32_t)v; memcpy((char*)p + 4 * i, &w, 4); break; }
    case O_INT64: case O_UINT64: memcpy((char*)p + 8 * i, &v, 8); break;
  }
}

static void o_reduce_elem(int dt, int op, const void* a, size_t ia, const void* b, size_t ib,
                          void* out, size_t io) {
  const int es = o_dtype_size(dt);
  if (op == O_AVG) op = O_SUM;   /* the hops of avg add; the final division is o_div_elem */
  if (o_is_int(dt)) {
    uint64_t x = o_geti(dt, a, ia), y = o_geti(dt, b, ib), r;
    int bgt, blt;   /* is the local operand strictly greater / smaller? */
    if (o_is_signed(dt)) { bgt = (int64_t)y > (int64_t)x; blt = (int64_t)y < (int64_t)x; }
    else { bgt = y > x; blt = y < x; }
    switch (op) {
      case O_SUM: r = x + y; break;                   /* wraps modulo 2^64, then to the width */
      case O_PROD: r = x * y; break;                  /* low bits of the product */
      case O_MAX: r = bgt ? y : x; break;             /* ties keep the received operand */
      default: r = blt ? y : x; break;                /* O_MIN */
    }
    o_puti(dt, out, io, r);
    return;
  }
  double x = o_get(dt, a, ia), y = o_get(dt, b, ib);
  if (op == O_SUM) {
    o_put(dt, out, io, x + y);
  } else if (op == O_PROD) {
    /* exact in double for fp32 / fp16 / bf16 operands (<= 48 significant
     * bits), so o_put rounds once; for fp64 the double product is the
     * correctly rounded one */
    o_put(dt, out, io, x * y);
  } else {
    /* select a bit pattern, no rounding: ties (including +0 == -0) keep a */
    int take_b = (op == O_MAX) ? (y > x) : (y < x);
    if (take_b) memcpy((char*)out + es * io, (const char*)b + es * ib, es);
    else memcpy((char*)out + es * io, (const char*)a + es * ia, es);
  }
}

/* avg's final step: element i of p divided by k (integers truncate toward
 * zero; floats round once to the dtype -- a double quotient rounded again is
 * innocuous, 53 >= 2p + 2) */
static void o_div_elem(int dt, void* p, size_t i, int k) {
  if (o_is_int(dt)) {
    uint64_t v = o_geti(dt, p, i);
    if (o_is_signed(dt)) o_puti(dt, p, i, (uint64_t)((int64_t)v / (int64_t)k));
    else o_puti(dt, p, i, v / (uint64_t)k);
    return;
  }
  o_put(dt, p, i, o_get(dt, p, i) / (double)k);
}

/* ------------------------------------------------------------------------ */
/* Partition [Sec. V-C]: channels -> outer loops -> chunks (reading R1).     */
/* ------------------------------------------------------------------------ */

/* data bytes one FIFO slot carries [Table "buffer sizes": Simple 512 KiB of
 * 512 KiB, LL 16 KiB of 32 KiB, LL128 562.5 KiB of 600 KiB] */
size_t o_slot_data_bytes(int proto, size_t slot_bytes) {
  switch (proto) {
    case O_SIMPLE: return slot_bytes;
    case O_LL: return slot_bytes / 2;               /* 4 data bytes per 8-byte line */
    case O_LL128: return (slot_bytes / 128) * 120;  /* 120 data bytes per 128-byte line */
  }
  return 0;
}

/* chunkCount in units (elements or bytes) for one elementary step */
size_t o_chunk_units(int proto, size_t slot_bytes, int chunk_steps, int unit_bytes) {
  size_t epp = 16 / (size_t)unit_bytes;
  size_t units = o_slot_data_bytes(proto, slot_bytes) * (size_t)chunk_steps / (size_t)unit_bytes;
  units = (units / epp) * epp;
  return units < epp ? epp : units;
}

/* workOffset / channelCount of channel ch among nch */
void o_channel_range(size_t n, int unit_bytes, int nch, int ch, size_t* start, size_t* len) {
  size_t epp = 16 / (size_t)unit_bytes;
  size_t npk = n / epp, tail = n % epp;
  size_t base = npk / (size_t)nch, rem = npk % (size_t)nch;
  size_t c = (size_t)ch;
  size_t sp = c * base + (c < rem ? c : rem);
  size_t lp = base + (c < rem ? 1 : 0);
  *start = sp * epp;
  *len = lp * epp + (ch == nch - 1 ? tail : 0);
}

/* segment s of one ring-AllReduce loop that starts at `off` inside a channel
 * ending at `end`: full loops use chunkCount, the last loop splits what is
 * left evenly over the k segments (rounded up to a pack) */
static size_t o_ceil_div(size_t a, size_t b) { return (a + b - 1) / b; }
size_t o_ring_loop_chunk(size_t off, size_t end, int k, size_t chunk, int unit_bytes) {
  size_t epp = 16 / (size_t)unit_bytes;
  size_t loop = (size_t)k * chunk;
  size_t rem = end - off;
  if (rem >= loop) return chunk;
  size_t c = o_ceil_div(rem, (size_t)k);
  return o_ceil_div(c, epp) * epp;
}

/* ------------------------------------------------------------------------ */
/* Step tables [Sec. V-E]                                                    */
/* ------------------------------------------------------------------------ */

/* Ring AllReduce, Table "Ring AllReduce": 0 send, 1..k-2 recvReduceSend,
 * k-1 recvReduceCopySend, k..2k-3 recvCopySend, 2k-2 recv */
int o_ring_allreduce_prim(int k, int t) {
  if (t == 0) return P_SEND;
  if (t <= k - 2) return P_RECV_REDUCE_SEND;
  if (t == k - 1) return P_RECV_REDUCE_COPY_SEND;
  if (t <= 2 * k - 3) return P_RECV_COPY_SEND;
  if (t == 2 * k - 2) return P_RECV;
  return P_NONE;
}
/* Ring ReduceScatter: 0 send, 1..k-2 recvReduceSend, k-1 recvReduceCopy */
int o_ring_reducescatter_prim(int k, int t) {
  if (t == 0) return P_SEND;
  if (t <= k - 2) return P_RECV_REDUCE_SEND;
  if (t == k - 1) return P_RECV_REDUCE_COPY;
  return P_NONE;
}
/* Ring AllGather: 0 send (in place) or copySend, 1..k-2 recvCopySend, k-1 recv */
int o_ring_allgather_prim(int k, int t, int inplace) {
  if (t == 0) return inplace ? P_SEND : P_COPY_SEND;
  if (t <= k - 2) return P_RECV_COPY_SEND;
  if (t == k - 1) return P_RECV;
  return P_NONE;
}
/* Ring Broadcast chain: root send / copySend, middle recvCopySend, last recv */
int o_bcast_prim(int k, int root, int r, int inplace) {
  int p = ((r - root) % k + k) % k;
  if (p == 0) return inplace ? P_SEND : P_COPY_SEND;
  if (p < k - 1) return P_RECV_COPY_SEND;
  return P_RECV;
}
/* Ring Reduce chain (reading R4): initiator root+1 send, middle
 * recvReduceSend, root recvReduceCopy */
int o_reduce_prim(int k, int root, int r) {
  int p = ((r - root - 1) % k + k) % k;
  if (p == 0) return P_SEND;
  if (p < k - 1) return P_RECV_REDUCE_SEND;
  return P_RECV_REDUCE_COPY;
}

/* ------------------------------------------------------------------------ */
/* Double binary tree [Sec. II-C] (reading R5).                              */
/* Tree A over 1-indexed nodes i = r + 1: odd nodes are leaves; node i with  */
/* lowest set bit b >= 2 has left child i - b/2 and as right child the first */
/* of i + b/2, i + b/4, ..., i + 1 that is <= k.  The root is the largest    */
/* power of two <= k.                                                        */
/* ------------------------------------------------------------------------ */
static int o_treeA_root(int k) { int p = 1; while (p * 2 <= k) p *= 2; return p; }
static void o_treeA_children(int k, int i, int* c0, int* c1) {
  *c0 = 0; *c1 = 0;
  if (i & 1) return;
  int b = i & -i;
  *c0 = i - b / 2;
  for (int d = b / 2; d >= 1; d /= 2) {
    if (i + d <= k) { *c1 = i + d; break; }
  }
}
/* rank that plays tree-A node i in tree `t` */
static int o_tree_rank_of_node(int k, int t, int i) {
  int ra = i - 1;                       /* rank playing node i in tree A */
  if (t == 0) return ra;
  if (k % 2 == 0) return k - 1 - ra;    /* mirror */
  return ((ra - 1) % k + k) % k;        /* shift: rank r plays the node of rank r+1 */
}
static int o_tree_node_of_rank(int k, int t, int r) {
  if (t == 0) return r + 1;
  if (k % 2 == 0) return (k - 1 - r) + 1;
  return ((r + 1) % k) + 1;
}
/* parent rank (-1 for the root) and children ranks (-1 for none), children
 * ordered by ascending tree-A node id */
void o_tree_links(int k, int t, int r, int* parent, int* child0, int* child1) {
  int i = o_tree_node_of_rank(k, t, r);
  *parent = -1; *child0 = -1; *child1 = -1;
  int c0, c1;
  o_treeA_children(k, i, &c0, &c1);
  if (c0) *child0 = o_tree_rank_of_node(k, t, c0);
  if (c1) *child1 = o_tree_rank_of_node(k, t, c1);
  for (int j = 1; j <= k; j++) {
    int a, b;
    o_treeA_children(k, j, &a, &b);
    if (a == i || b == i) { *parent = o_tree_rank_of_node(k, t, j); break; }
  }
}
int o_tree_root(int k, int t) { return o_tree_rank_of_node(k, t, o_treeA_root(k)); }

/* ------------------------------------------------------------------------ */
/* Hierarchical tree [Sec. V-E: the branching structure is built only across */
/* nodes; inside each node the ranks form a simple chain] (reading R19).     */
/* The k ranks form k/m nodes of m consecutive ranks; the double binary tree */
/* above links the nodes.  Inside node n the chain runs n*m -> n*m+1 -> ...  */
/* -> n*m+m-1 downwards: the first rank of a node hangs from the last rank   */
/* of its parent node, and the last rank of a node carries the node's child  */
/* nodes (their first ranks, in tree-A node order), so no rank has more than */
/* two children.  m = 1 is the flat tree.                                    */
/* ------------------------------------------------------------------------ */
void o_htree_links(int k, int m, int t, int r, int* parent, int* child0, int* child1) {
  if (m <= 1) { o_tree_links(k, t, r, parent, child0, child1); return; }
  int nn = k / m, node = r / m, i = r % m;
  int pn = -1, c0 = -1, c1 = -1;
  if (nn > 1) o_tree_links(nn, t, node, &pn, &c0, &c1);
  *parent = (i > 0) ? r - 1 : (pn >= 0 ? pn * m + m - 1 : -1);
  if (i < m - 1) { *child0 = r + 1; *child1 = -1; }
  else { *child0 = c0 >= 0 ? c0 * m : -1; *child1 = c1 >= 0 ? c1 * m : -1; }
}
int o_htree_root(int k, int m, int t) {
  if (m <= 1) return o_tree_root(k, t);
  int nn = k / m;
  return (nn > 1 ? o_tree_root(nn, t) : 0) * m;
}

/* Tree AllReduce roles, Table "Tree AllReduce": root recvReduceCopySend;
 * middle recvReduceSend then recvCopySend; leaf send then recv */
void o_tree_prims(int k, int t, int r, int* up, int* down) {
  int p, c0, c1;
  o_tree_links(k, t, r, &p, &c0, &c1);
  if (p < 0) { *up = P_RECV_REDUCE_COPY_SEND; *down = P_NONE; }
  else if (c0 >= 0) { *up = P_RECV_REDUCE_SEND; *down = P_RECV_COPY_SEND; }
  else { *up = P_SEND; *down = P_RECV; }
}

/* ------------------------------------------------------------------------ */
/* Primitive executor: one elementary step of one rank on n units.           */
/* recv = FIFO contents from the predecessor, local = user input, out = user */
/* output, fifo_out = what goes to the successor.                            */
/* ------------------------------------------------------------------------ */
static void o_exec(int prim, int dt, int op, int k, size_t n, const void* recv, const void* local,
                   void* out, void* fifo_out) {
  int es = o_dtype_size(dt);
  size_t nb = n * (size_t)es;
  switch (prim) {
    case P_SEND:
      memcpy(fifo_out, local, nb);
      break;
    case P_COPY_SEND:
      memcpy(out, local, nb);
      memcpy(fifo_out, local, nb);
      break;
    case P_RECV:
      memcpy(out, recv, nb);
      break;
    case P_RECV_COPY_SEND:
      memcpy(out, recv, nb);
      memcpy(fifo_out, recv, nb);
      break;
    case P_RECV_REDUCE_SEND:
      for (size_t i = 0; i < n; i++) o_reduce_elem(dt, op, recv, i, local, i, fifo_out, i);
      break;
    case P_RECV_REDUCE_COPY:
      for (size_t i = 0; i < n; i++) o_reduce_elem(dt, op, recv, i, local, i, out, i);
      if (op == O_AVG) for (size_t i = 0; i < n; i++) o_div_elem(dt, out, i, k);
      break;
    case P_RECV_REDUCE_COPY_SEND:
      /* the step that completes a value writes it and forwards it: avg
       * divides here, once */
      for (size_t i = 0; i < n; i++) o_reduce_elem(dt, op, recv, i, local, i, out, i);
      if (op == O_AVG) for (size_t i = 0; i < n; i++) o_div_elem(dt, out, i, k);
      memcpy(fifo_out, out, nb);
      break;
    default:
      break;
  }
}

static int o_mod(int a, int k) { return ((a % k) + k) % k; }

/* ------------------------------------------------------------------------ */
/* Ring AllReduce [Sec. V-E, Table "Ring AllReduce"] (readings R1-R3).       */
/* send[r], recv[r]: count elements each.  Returns 0 on success.             */
/* ------------------------------------------------------------------------ */
int o_ring_allreduce(int k, int nch, size_t chunk, int dt, int op, size_t count,
                     const void* const* send, void* const* recv) {
  int es = o_dtype_size(dt);
  if (k < 1 || nch < 1 || es == 0 || chunk == 0) return -1;
  if (k == 1) { memcpy(recv[0], send[0], count * (size_t)es); return 0; }
  char** fprev = calloc((size_t)k, sizeof(char*));
  char** fnext = calloc((size_t)k, sizeof(char*));
  for (int r = 0; r < k; r++) {
    fprev[r] = malloc(chunk * (size_t)es + 16);
    fnext[r] = malloc(chunk * (size_t)es + 16);
  }
  for (int ch = 0; ch < nch; ch++) {
    size_t start, len;
    o_channel_range(count, es, nch, ch, &start, &len);
    size_t end = start + len;
    size_t loop = (size_t)k * chunk;
    for (size_t off = start; off < end; off += loop) {
      size_t c = o_ring_loop_chunk(off, end, k, chunk, es);
      for (int t = 0; t <= 2 * k - 2; t++) {
        int prim = o_ring_allreduce_prim(k, t);
        for (int r = 0; r < k; r++) {
          int s = o_mod(r - t - 1, k);
          size_t a = off + (size_t)s * c;
          if (a > end) a = end;
          size_t b = a + c;
          if (b > end) b = end;
          size_t n = b - a;
          o_exec(prim, dt, op, k, n, fprev[o_mod(r - 1, k)], (const char*)send[r] + a * es,
                 (char*)recv[r] + a * es, fnext[r]);
        }
        char** tmp = fprev; fprev = fnext; fnext = tmp;
      }
    }
  }
  for (int r = 0; r < k; r++) { free(fprev[r]); free(fnext[r]); }
  free(fprev); free(fnext);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Ring ReduceScatter [Table "Ring ReduceScatter"].  send[r] holds k blocks  */
/* of recvcount elements; block b is reduced onto rank b.                    */
/* ------------------------------------------------------------------------ */
int o_ring_reducescatter(int k, int nch, size_t chunk, int dt, int op, size_t recvcount,
                         const void* const* send, void* const* recv) {
  int es = o_dtype_size(dt);
  if (k < 1 || nch < 1 || es == 0 || chunk == 0) return -1;
  if (k == 1) { memcpy(recv[0], send[0], recvcount * (size_t)es); return 0; }
  char** fprev = calloc((size_t)k, sizeof(char*));
  char** fnext = calloc((size_t)k, sizeof(char*));
  for (int r = 0; r < k; r++) {
    fprev[r] = malloc(chunk * (size_t)es + 16);
    fnext[r] = malloc(chunk * (size_t)es + 16);
  }
  for (int ch = 0; ch < nch; ch++) {
    size_t start, len;
    o_channel_range(recvcount, es, nch, ch, &start, &len);
    size_t end = start + len;
    for (size_t off = start; off < end; off += chunk) {
      size_t n = (end - off < chunk) ? end - off : chunk;
      for (int t = 0; t <= k - 1; t++) {
        int prim = o_ring_reducescatter_prim(k, t);
        for (int r = 0; r < k; r++) {
          int s = o_mod(r - t - 1, k);
          size_t a = (size_t)s * recvcount + off;
          o_exec(prim, dt, op, k, n, fprev[o_mod(r - 1, k)], (const char*)send[r] + a * es,
                 (char*)recv[r] + off * es, fnext[r]);
        }
        char** tmp = fprev; fprev = fnext; fnext = tmp;
      }
    }
  }
  for (int r = 0; r < k; r++) { free(fprev[r]); free(fnext[r]); }
  free(fprev); free(fnext);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Ring AllGather [Table "Ring AllGather"], byte units [Sec. V-C].           */
/* send[r] holds nbytes; recv[r] holds k blocks of nbytes.                   */
/* ------------------------------------------------------------------------ */
int o_ring_allgather(int k, int nch, size_t chunk, size_t nbytes,
                     const void* const* send, void* const* recv) {
  if (k < 1 || nch < 1 || chunk == 0) return -1;
  char** fprev = calloc((size_t)k, sizeof(char*));
  char** fnext = calloc((size_t)k, sizeof(char*));
  for (int r = 0; r < k; r++) { fprev[r] = malloc(chunk + 16); fnext[r] = malloc(chunk + 16); }
  for (int ch = 0; ch < nch; ch++) {
    size_t start, len;
    o_channel_range(nbytes, 1, nch, ch, &start, &len);
    size_t end = start + len;
    for (size_t off = start; off < end; off += chunk) {
      size_t n = (end - off < chunk) ? end - off : chunk;
      for (int t = 0; t <= k - 1; t++) {
        /* the oracle always uses distinct buffers, so step 0 is copySend */
        int prim = (k == 1) ? P_COPY_SEND : o_ring_allgather_prim(k, t, 0);
        for (int r = 0; r < k; r++) {
          int blk = o_mod(r - t, k);
          o_exec(prim, O_BYTE, O_SUM, k, n, fprev[o_mod(r - 1, k)], (const char*)send[r] + off,
                 (char*)recv[r] + (size_t)blk * nbytes + off, fnext[r]);
        }
        char** tmp = fprev; fprev = fnext; fnext = tmp;
      }
    }
  }
  for (int r = 0; r < k; r++) { free(fprev[r]); free(fnext[r]); }
  free(fprev); free(fnext);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Ring Broadcast [Table "Ring Broadcast"], byte units; chain from the root. */
/* ------------------------------------------------------------------------ */
int o_ring_broadcast(int k, int nch, size_t chunk, size_t nbytes, int root,
                     const void* const* send, void* const* recv) {
  if (k < 1 || nch < 1 || chunk == 0 || root < 0 || root >= k) return -1;
  char* fifo = malloc(chunk + 16);
  char* fifo2 = malloc(chunk + 16);
  for (int ch = 0; ch < nch; ch++) {
    size_t start, len;
    o_channel_range(nbytes, 1, nch, ch, &start, &len);
    size_t end = start + len;
    for (size_t off = start; off < end; off += chunk) {
      size_t n = (end - off < chunk) ? end - off : chunk;
      for (int p = 0; p < k; p++) {           /* walk the chain root, root+1, ... */
        int r = o_mod(root + p, k);
        int prim = (k == 1) ? P_COPY_SEND : o_bcast_prim(k, root, r, 0);
        o_exec(prim, O_BYTE, O_SUM, k, n, fifo, (const char*)send[r] + off, (char*)recv[r] + off,
               fifo2);
        char* tmp = fifo; fifo = fifo2; fifo2 = tmp;
      }
    }
  }
  free(fifo); free(fifo2);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Ring Reduce [Table "Ring Reduce"]: chain root+1 -> ... -> root.           */
/* Only recv[root] is written.                                               */
/* ------------------------------------------------------------------------ */
int o_ring_reduce(int k, int nch, size_t chunk, int dt, int op, size_t count, int root,
                  const void* const* send, void* const* recv) {
  int es = o_dtype_size(dt);
  if (k < 1 || nch < 1 || es == 0 || chunk == 0 || root < 0 || root >= k) return -1;
  if (k == 1) { memcpy(recv[0], send[0], count * (size_t)es); return 0; }
  char* fifo = malloc(chunk * (size_t)es + 16);
  char* fifo2 = malloc(chunk * (size_t)es + 16);
  for (int ch = 0; ch < nch; ch++) {
    size_t start, len;
    o_channel_range(count, es, nch, ch, &start, &len);
    size_t end = start + len;
    for (size_t off = start; off < end; off += chunk) {
      size_t n = (end - off < chunk) ? end - off : chunk;
      for (int p = 0; p < k; p++) {           /* walk the chain root+1, ..., root */
        int r = o_mod(root + 1 + p, k);
        int prim = o_reduce_prim(k, root, r);
        o_exec(prim, dt, op, k, n, fifo, (const char*)send[r] + off * es,
               recv[r] ? (char*)recv[r] + off * es : NULL, fifo2);
        char* tmp = fifo; fifo = fifo2; fifo2 = tmp;
      }
    }
  }
  free(fifo); free(fifo2);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Tree AllReduce [Sec. V-E, Table "Tree AllReduce"] on the double binary    */
/* tree.  Reduce phase: every rank sends up f(child1, f(child0, own)), the   */
/* root writes the result; broadcast phase: the result is copied down.       */
/* ------------------------------------------------------------------------ */
typedef struct {
  int k, m, t, dt, op;
  size_t n, off;
  const void* const* send;
  char** val;               /* per rank: value sent up (n units) */
} OTreeCtx;

static void o_tree_up(OTreeCtx* c, int r) {
  int es = o_dtype_size(c->dt);
  int p, c0, c1;
  o_htree_links(c->k, c->m, c->t, r, &p, &c0, &c1);
  const char* own = (const char*)c->send[r] + c->off * es;
  memcpy(c->val[r], own, c->n * (size_t)es);
  int kids[2] = {c0, c1};
  for (int j = 0; j < 2; j++) {
    if (kids[j] < 0) continue;
    o_tree_up(c, kids[j]);
    for (size_t i = 0; i < c->n; i++)
      o_reduce_elem(c->dt, c->op, c->val[kids[j]], i, c->val[r], i, c->val[r], i);
  }
}

int o_tree_allreduce_m(int k, int m, int nch, size_t chunk, int dt, int op, size_t count,
                       const void* const* send, void* const* recv) {
  int es = o_dtype_size(dt);
  if (k < 1 || nch < 1 || es == 0 || chunk == 0 || m < 1 || k % m) return -1;
  if (k == 1) { memcpy(recv[0], send[0], count * (size_t)es); return 0; }
  char** val = calloc((size_t)k, sizeof(char*));
  for (int r = 0; r < k; r++) val[r] = malloc(chunk * (size_t)es + 16);
  int nsub = 2 * nch;          /* each channel's data: first half tree A, second half tree B */
  for (int j = 0; j < nsub; j++) {
    int t = j % 2;
    size_t start, len;
    o_channel_range(count, es, nsub, j, &start, &len);
    size_t end = start + len;
    for (size_t off = start; off < end; off += chunk) {
      size_t n = (end - off < chunk) ? end - off : chunk;
      OTreeCtx c = {k, m, t, dt, op, n, off, send, val};
      int root = o_htree_root(k, m, t);
      o_tree_up(&c, root);
      /* the root's recvReduceCopySend completes the value (avg divides) */
      if (op == O_AVG) for (size_t i = 0; i < n; i++) o_div_elem(dt, val[root], i, k);
      for (int r = 0; r < k; r++) memcpy((char*)recv[r] + off * es, val[root], n * (size_t)es);
    }
  }
  for (int r = 0; r < k; r++) free(val[r]);
  free(val);
  return 0;
}

int o_tree_allreduce(int k, int nch, size_t chunk, int dt, int op, size_t count,
                     const void* const* send, void* const* recv) {
  return o_tree_allreduce_m(k, 1, nch, chunk, dt, op, count, send, recv);
}

/* ------------------------------------------------------------------------ */
/* LL and LL128 line encodings [Sec. III-B, III-C]                           */
/* LL: one 8-byte line = (flag << 32) | 4 data bytes, little endian.         */
/* LL128: one 128-byte line = 16 words; words 0..14 carry 120 data bytes in  */
/* order, word 15 carries the 64-bit flag.  Partial tails are zero padded.   */
/* ------------------------------------------------------------------------ */
size_t o_ll_lines(size_t nbytes) { return o_ceil_div(nbytes, 4); }
size_t o_ll128_lines(size_t nbytes) { return o_ceil_div(nbytes, 120); }

void o_ll_encode(const uint8_t* data, size_t nbytes, uint32_t flag, uint64_t* lines) {
  size_t nl = o_ll_lines(nbytes);
  for (size_t l = 0; l < nl; l++) {
    uint32_t d = 0;
    for (int b = 0; b < 4; b++) {
      size_t i = 4 * l + (size_t)b;
      if (i < nbytes) d |= (uint32_t)data[i] << (8 * b);
    }
    lines[l] = ((uint64_t)flag << 32) | d;
  }
}
/* returns 0, or 1 + index of the first line whose flag is not `flag` */
long o_ll_decode(const uint64_t* lines, size_t nbytes, uint32_t flag, uint8_t* data) {
  size_t nl = o_ll_lines(nbytes);
  for (size_t l = 0; l < nl; l++) {
    if ((uint32_t)(lines[l] >> 32) != flag) return (long)l + 1;
    uint32_t d = (uint32_t)lines[l];
    for (int b = 0; b < 4; b++) {
      size_t i = 4 * l + (size_t)b;
      if (i < nbytes) data[i] = (uint8_t)(d >> (8 * b));
    }
  }
  return 0;
}
void o_ll128_encode(const uint8_t* data, size_t nbytes, uint64_t flag, uint64_t* lines) {
  size_t nl = o_ll128_lines(nbytes);
  for (size_t l = 0; l < nl; l++) {
    uint8_t* line = (uint8_t*)(lines + 16 * l);
    for (int b = 0; b < 120; b++) {
      size_t i = 120 * l + (size_t)b;
      line[b] = (i < nbytes) ? data[i] : 0;
    }
    lines[16 * l + 15] = flag;
  }
}
long o_ll128_decode(const uint64_t* lines, size_t nbytes, uint64_t flag, uint8_t* data) {
  size_t nl = o_ll128_lines(nbytes);
  for (size_t l = 0; l < nl; l++) {
    if (lines[16 * l + 15] != flag) return (long)l + 1;
    const uint8_t* line = (const uint8_t*)(lines + 16 * l);
    for (int b = 0; b < 120; b++) {
      size_t i = 120 * l + (size_t)b;
      if (i < nbytes) data[i] = line[b];
    }
  }
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Point queries: the value of ONE output element, for sampled checks of     */
/* outputs too large to replay whole.  vals[r] is element i of rank r's      */
/* input (dtype dt).  They follow the same partition and fold orders as the  */
/* full replays above (which the tests check element by element).            */
/* ------------------------------------------------------------------------ */

/* ring AllReduce: segment s of the loop holding i is folded x_{s+1}, ..., x_s */
int o_ring_allreduce_point(int k, int nch, size_t chunk, int dt, int op, size_t count, size_t i,
                           const void* vals, void* out) {
  int es = o_dtype_size(dt);
  if (k < 1 || i >= count) return -1;
  if (k == 1) { memcpy(out, vals, (size_t)es); return 0; }
  for (int ch = 0; ch < nch; ch++) {
    size_t start, len;
    o_channel_range(count, es, nch, ch, &start, &len);
    if (i < start || i >= start + len) continue;
    size_t end = start + len, loop = (size_t)k * chunk;
    size_t off = start + ((i - start) / loop) * loop;
    size_t c = o_ring_loop_chunk(off, end, k, chunk, es);
    int s = (int)((i - off) / c);
    char acc[8];
    memcpy(acc, (const char*)vals + (size_t)es * (size_t)o_mod(s + 1, k), (size_t)es);
    for (int m = 2; m <= k; m++) {
      int r = o_mod(s + m, k);
      o_reduce_elem(dt, op, acc, 0, vals, (size_t)r, acc, 0);
    }
    if (op == O_AVG) o_div_elem(dt, acc, 0, k);
    memcpy(out, acc, (size_t)es);
    return 0;
  }
  return -1;
}

/* tree AllReduce: sub-channel j holding i runs tree j % 2 */
static void o_tree_point_up(int k, int m, int t, int dt, int op, int r, const void* vals, char* out) {
  int es = o_dtype_size(dt);
  int p, c0, c1;
  o_htree_links(k, m, t, r, &p, &c0, &c1);
  memcpy(out, (const char*)vals + (size_t)es * (size_t)r, (size_t)es);
  int kids[2] = {c0, c1};
  for (int j = 0; j < 2; j++) {
    if (kids[j] < 0) continue;
    char sub[8];
    o_tree_point_up(k, m, t, dt, op, kids[j], vals, sub);
    o_reduce_elem(dt, op, sub, 0, out, 0, out, 0);
  }
}
int o_tree_allreduce_point_m(int k, int m, int nch, size_t chunk, int dt, int op, size_t count,
                             size_t i, const void* vals, void* out) {
  int es = o_dtype_size(dt);
  (void)chunk;
  if (k < 1 || i >= count || m < 1 || k % m) return -1;
  if (k == 1) { memcpy(out, vals, (size_t)es); return 0; }
  int nsub = 2 * nch;
  for (int j = 0; j < nsub; j++) {
    size_t start, len;
    o_channel_range(count, es, nsub, j, &start, &len);
    if (i < start || i >= start + len) continue;
    char acc[8];
    o_tree_point_up(k, m, j % 2, dt, op, o_htree_root(k, m, j % 2), vals, acc);
    if (op == O_AVG) o_div_elem(dt, acc, 0, k);
    memcpy(out, acc, (size_t)es);
    return 0;
  }
  return -1;
}
int o_tree_allreduce_point(int k, int nch, size_t chunk, int dt, int op, size_t count, size_t i,
                           const void* vals, void* out) {
  return o_tree_allreduce_point_m(k, 1, nch, chunk, dt, op, count, i, vals, out);
}

/* ring ReduceScatter: element i of rank b's output folds block b in the
 * order x_{b+1}, ..., x_b (the partition does not change the order) */
int o_ring_reducescatter_point(int k, int dt, int op, int b, const void* vals, void* out) {
  int es = o_dtype_size(dt);
  if (k < 1 || b < 0 || b >= k) return -1;
  char acc[8];
  memcpy(acc, (const char*)vals + (size_t)es * (size_t)o_mod(b + 1, k), (size_t)es);
  for (int m = 2; m <= k; m++) o_reduce_elem(dt, op, acc, 0, vals, (size_t)o_mod(b + m, k), acc, 0);
  if (op == O_AVG && k > 1) o_div_elem(dt, acc, 0, k);
  memcpy(out, acc, (size_t)es);
  return 0;
}

/* ring Reduce: the chain root+1, ..., root */
int o_ring_reduce_point(int k, int dt, int op, int root, const void* vals, void* out) {
  int es = o_dtype_size(dt);
  if (k < 1 || root < 0 || root >= k) return -1;
  char acc[8];
  memcpy(acc, (const char*)vals + (size_t)es * (size_t)o_mod(root + 1, k), (size_t)es);
  for (int m = 2; m <= k; m++) o_reduce_elem(dt, op, acc, 0, vals, (size_t)o_mod(root + m, k), acc, 0);
  if (op == O_AVG && k > 1) o_div_elem(dt, acc, 0, k);
  memcpy(out, acc, (size_t)es);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* All-to-all [Sec. II-A-4: a group of Send/Recv calls emulating All-to-All]:
 * block j (block_bytes) of rank r's input is received by rank j as its
 * block r.  Byte loops; no arithmetic. */
/* ------------------------------------------------------------------------ */
int o_alltoall(int k, size_t block_bytes, const unsigned char* const* in, unsigned char* const* out) {
  if (k < 1) return -1;
  for (int r = 0; r < k; r++)
    for (int j = 0; j < k; j++)
      for (size_t b = 0; b < block_bytes; b++)
        out[j][(size_t)r * block_bytes + b] = in[r][(size_t)j * block_bytes + b];
  return 0;
}
