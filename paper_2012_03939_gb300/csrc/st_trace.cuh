// Stack-based traversal of the 4-wide BVH (closest hit and any hit).
//
// The binary LBVH (internal node = 64 bytes: both child boxes, then the two
// child links) is collapsed into 4-wide nodes of 112 bytes, seven float4 read
// as 16-byte vector loads: lo.x, hi.x, lo.y, hi.y, lo.z, hi.z of the four
// children, then the four child links. Leaf i is the triangle record
// tri[3i..3i+2] = v0 (w = face id bits), v1, v2, stored in Morton order.
// The first TRACE_SH entries of the stack live in shared memory (strided by
// block size), the rest in local memory.
#pragma once
#include "st_device.cuh"

namespace st {

constexpr int TRACE_SH = 16;
constexpr int TRACE_DEPTH = 96;   // 4-wide nodes push up to three children per level
constexpr int ERR_STACK = 1;
constexpr int ERR_LOOP = 2;   // more node fetches than the tree has nodes, or a node index past them
constexpr int ERR_INDEX = 8;  // a leaf or bin-list index outside its array (the access is skipped)

struct TraceStats { int visits, tests; };

__device__ __forceinline__ float3 safe_inv(float3 d) {
  auto inv1 = [](float x) { return fabsf(x) > 1e-30f ? 1.0f / x : copysignf(1e30f, x); };
  return mk3(inv1(d.x), inv1(d.y), inv1(d.z));
}

// slab test of box [lo, hi]; returns entry distance or +inf on a miss
__device__ __forceinline__ float box_hit(float lx, float hx, float ly, float hy, float lz, float hz, float3 o,
                                         float3 inv, float tmax) {
  float tx0 = (lx - o.x) * inv.x, tx1 = (hx - o.x) * inv.x;
  float ty0 = (ly - o.y) * inv.y, ty1 = (hy - o.y) * inv.y;
  float tz0 = (lz - o.z) * inv.z, tz1 = (hz - o.z) * inv.z;
  float tn = fmaxf(fmaxf(fminf(tx0, tx1), fminf(ty0, ty1)), fmaxf(fminf(tz0, tz1), 0.0f));
  float tf = fminf(fminf(fmaxf(tx0, tx1), fmaxf(ty0, ty1)), fminf(fmaxf(tz0, tz1), tmax));
  // widen the far distance by 1 + 2*gamma(3) so rounding never culls a hit
  // (Ize, "Robust BVH Ray Traversal", JCGT 2013)
  return tn <= tf * 1.00000036f ? tn : __int_as_float(0x7f800000);
}

// ANY = stop at the first hit (shadow rays). nf = leaves (faces), nn = 4-wide
// nodes: indices outside them latch an error bit. Returns the face id or -1; t in
// tbest; the hit's leaf index in *leaf_out if given. EX2 = a second face
// (exclude2) is skipped too.
// nodes = the 4-wide tree: per node lo.x, hi.x, lo.y, hi.y, lo.z, hi.z (one
// float4 of four children each) and the four child links (>= 0 node, < 0 leaf
// ~i, INT_MIN empty). Hit leaves are tested at once; hit internal children are
// sorted by entry distance, the nearest is visited next, the others pushed.
template <bool ANY, bool STATS, bool EX2 = false>
__device__ __forceinline__ int trace_bvh(const float4* __restrict__ nodes, const float4* __restrict__ tri, int nf,
                                         int nn, float3 o, float3 d, float tmax, int exclude, float& tbest, int* sstack,
                                         int* err, TraceStats* ts, int* leaf_out = nullptr, int exclude2 = -1) {
  RayPre rp = ray_pre(o, d);
  float3 inv = safe_inv(d);
  int best = -1, best_leaf = -1;
  tbest = tmax;
  auto leaf = [&](int li) -> bool {
    if ((unsigned)li >= (unsigned)nf) { atomicOr(err, ERR_INDEX); return false; }
    float4 a = __ldg(&tri[3 * li]);
    int fid = __float_as_int(a.w);
    if (STATS) ts->tests++;
    if (fid == exclude || (EX2 && fid == exclude2)) return false;
    float4 b = __ldg(&tri[3 * li + 1]);
    float4 c = __ldg(&tri[3 * li + 2]);
    float t = tri_test(rp, xyz(a), xyz(b), xyz(c), ANY ? tmax : tbest * 1.0000001f + 1e-30f);
    if (t > 0.0f) {
      if (ANY) { best = fid; best_leaf = li; tbest = t; return true; }
      if (t < tbest || (t == tbest && fid < best)) { tbest = t; best = fid; best_leaf = li; }
    }
    return false;
  };
  if (nf == 1) {
    leaf(0);
    if (leaf_out) *leaf_out = best_leaf;
    return best;
  }
  const float INF = __int_as_float(0x7f800000);
  const int EMPTY = (int)0x80000000;
  int local[TRACE_DEPTH - TRACE_SH];
  const int bd = blockDim.x;
  int sp = 0;
  int node = 0;
  int budget = nn;  // a well-formed tree fetches each of its nn nodes at most once
  for (;;) {
    if (--budget < 0 || (unsigned)node >= (unsigned)nn) { atomicOr(err, ERR_LOOP); return best; }
    const float4* np = nodes + 7 * node;
    float4 lx = __ldg(np), hx = __ldg(np + 1), ly = __ldg(np + 2), hy = __ldg(np + 3), lz = __ldg(np + 4),
           hz = __ldg(np + 5), ch = __ldg(np + 6);
    if (STATS) ts->visits++;
    int c[4] = {__float_as_int(ch.x), __float_as_int(ch.y), __float_as_int(ch.z), __float_as_int(ch.w)};
    float t[4];
    t[0] = box_hit(lx.x, hx.x, ly.x, hy.x, lz.x, hz.x, o, inv, tbest);
    t[1] = box_hit(lx.y, hx.y, ly.y, hy.y, lz.y, hz.y, o, inv, tbest);
    t[2] = box_hit(lx.z, hx.z, ly.z, hy.z, lz.z, hz.z, o, inv, tbest);
    t[3] = box_hit(lx.w, hx.w, ly.w, hy.w, lz.w, hz.w, o, inv, tbest);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      if (c[j] == EMPTY) t[j] = INF;
      if (c[j] < 0 && t[j] != INF) {
        if (leaf(~c[j]) && ANY) return best;
        t[j] = INF;
      }
    }
    // internal children still in front of the current hit, nearest first
#pragma unroll
    for (int j = 0; j < 4; ++j)
      if (t[j] > tbest * 1.00000036f) t[j] = INF;
    auto cswap = [&](int a, int b) {
      if (t[b] < t[a]) {
        float tt = t[a]; t[a] = t[b]; t[b] = tt;
        int cc = c[a]; c[a] = c[b]; c[b] = cc;
      }
    };
    cswap(0, 1); cswap(2, 3); cswap(0, 2); cswap(1, 3); cswap(1, 2);
    if (t[0] == INF) {
      if (sp == 0) break;
      --sp;
      node = sp < TRACE_SH ? sstack[sp * bd] : local[sp - TRACE_SH];
      continue;
    }
    node = c[0];
#pragma unroll
    for (int j = 3; j >= 1; --j) {
      if (t[j] == INF) continue;
      if (sp >= TRACE_DEPTH) { atomicOr(err, ERR_STACK); return best; }
      if (sp < TRACE_SH) sstack[sp * bd] = c[j]; else local[sp - TRACE_SH] = c[j];
      ++sp;
    }
  }
  if (leaf_out) *leaf_out = best_leaf;
  return best;
}

}  // namespace st
