// LBVH construction and refit.
//
// Build: centroid bounds -> 30-bit Morton code per triangle centroid -> stable
// LSD radix sort of (code, face id) -> a hierarchy over the leaves in that
// order: Karras' parallel radix tree ("Maximizing Parallelism in the
// Construction of BVHs, Octrees, and k-d Trees", HPG 2012; ties between equal
// codes broken by the leaf index), or PLOC clustering (below: trees of lower
// surface-area cost for a few more milliseconds) -> leaf triangle records in
// Morton order -> boxes bottom-up, the second thread to reach a node merging
// its two children. Refit reuses the order and the hierarchy: new vertex
// positions only rewrite the leaf records and the boxes.
#include <algorithm>
#include <cstdio>

#include "st_internal.h"

namespace st {
namespace {

constexpr int RS_THREADS = 256;
constexpr int RS_ROUNDS = 16;
constexpr int RS_TILE = RS_THREADS * RS_ROUNDS;

__device__ __forceinline__ int ordered(float f) {
  int i = __float_as_int(f);
  return i >= 0 ? i : i ^ 0x7fffffff;
}
__device__ __forceinline__ float unordered(int i) { return __int_as_float(i >= 0 ? i : i ^ 0x7fffffff); }

__device__ __forceinline__ float3 centroid(const float* V, const int* F, int f) {
  int a = F[3 * f], b = F[3 * f + 1], c = F[3 * f + 2];
  return mk3((V[3 * a] + V[3 * b] + V[3 * c]) * (1.0f / 3.0f), (V[3 * a + 1] + V[3 * b + 1] + V[3 * c + 1]) * (1.0f / 3.0f),
             (V[3 * a + 2] + V[3 * b + 2] + V[3 * c + 2]) * (1.0f / 3.0f));
}

__global__ void k_init_bounds(int* b) {
  if (threadIdx.x < 3) b[threadIdx.x] = 0x7fffffff;
  else if (threadIdx.x < 6) b[threadIdx.x] = (int)0x80000000;
}

__global__ void k_centroid_bounds(const float* V, const int* F, int nf, int* bounds) {
  float3 lo = mk3(3.4e38f, 3.4e38f, 3.4e38f), hi = mk3(-3.4e38f, -3.4e38f, -3.4e38f);
  for (int f = blockIdx.x * blockDim.x + threadIdx.x; f < nf; f += gridDim.x * blockDim.x) {
    float3 c = centroid(V, F, f);
    lo = mk3(fminf(lo.x, c.x), fminf(lo.y, c.y), fminf(lo.z, c.z));
    hi = mk3(fmaxf(hi.x, c.x), fmaxf(hi.y, c.y), fmaxf(hi.z, c.z));
  }
  for (int off = 16; off > 0; off >>= 1) {
    lo.x = fminf(lo.x, __shfl_xor_sync(0xffffffffu, lo.x, off));
    lo.y = fminf(lo.y, __shfl_xor_sync(0xffffffffu, lo.y, off));
    lo.z = fminf(lo.z, __shfl_xor_sync(0xffffffffu, lo.z, off));
    hi.x = fmaxf(hi.x, __shfl_xor_sync(0xffffffffu, hi.x, off));
    hi.y = fmaxf(hi.y, __shfl_xor_sync(0xffffffffu, hi.y, off));
    hi.z = fmaxf(hi.z, __shfl_xor_sync(0xffffffffu, hi.z, off));
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMin(&bounds[0], ordered(lo.x)); atomicMin(&bounds[1], ordered(lo.y)); atomicMin(&bounds[2], ordered(lo.z));
    atomicMax(&bounds[3], ordered(hi.x)); atomicMax(&bounds[4], ordered(hi.y)); atomicMax(&bounds[5], ordered(hi.z));
  }
}

__device__ __forceinline__ uint32_t spread10(uint32_t v) {
  v = (v * 0x00010001u) & 0xFF0000FFu;
  v = (v * 0x00000101u) & 0x0F00F00Fu;
  v = (v * 0x00000011u) & 0xC30C30C3u;
  v = (v * 0x00000005u) & 0x49249249u;
  return v;
}

__global__ void k_morton(const float* V, const int* F, int nf, const int* bounds, uint32_t* keys, int* ids) {
  int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= nf) return;
  float3 lo = mk3(unordered(bounds[0]), unordered(bounds[1]), unordered(bounds[2]));
  float3 hi = mk3(unordered(bounds[3]), unordered(bounds[4]), unordered(bounds[5]));
  float3 c = centroid(V, F, f);
  float3 ext = hi - lo;
  auto q = [](float x, float l, float e) -> uint32_t {
    float u = e > 0.0f ? (x - l) / e : 0.5f;
    return (uint32_t)fminf(fmaxf(u * 1024.0f, 0.0f), 1023.0f);
  };
  keys[f] = (spread10(q(c.x, lo.x, ext.x)) << 2) | (spread10(q(c.y, lo.y, ext.y)) << 1) | spread10(q(c.z, lo.z, ext.z));
  ids[f] = f;
}

// ---- stable LSD radix sort, 8-bit digits
__global__ void k_rs_hist(const uint32_t* keys, int n, int shift, uint32_t* hist, int nblk) {
  __shared__ uint32_t h[256];
  h[threadIdx.x] = 0;
  __syncthreads();
  int base = blockIdx.x * RS_TILE;
  for (int i = threadIdx.x; i < RS_TILE; i += RS_THREADS) {
    int idx = base + i;
    if (idx < n) atomicAdd(&h[(keys[idx] >> shift) & 255u], 1u);
  }
  __syncthreads();
  hist[threadIdx.x * nblk + blockIdx.x] = h[threadIdx.x];
}

// exclusive scan of m counters in place, one block of 1024 threads
__global__ void k_rs_scan(uint32_t* hist, int m) {
  __shared__ uint32_t part[1024];
  int per = (m + 1023) / 1024;
  int b = threadIdx.x * per, e = min(b + per, m);
  uint32_t s = 0;
  for (int i = b; i < e; ++i) s += hist[i];
  part[threadIdx.x] = s;
  __syncthreads();
  for (int off = 1; off < 1024; off <<= 1) {
    uint32_t v = threadIdx.x >= off ? part[threadIdx.x - off] : 0;
    __syncthreads();
    part[threadIdx.x] += v;
    __syncthreads();
  }
  uint32_t run = part[threadIdx.x] - s;
  for (int i = b; i < e; ++i) { uint32_t c = hist[i]; hist[i] = run; run += c; }
}

__global__ void k_rs_scatter(const uint32_t* kin, const int* iin, uint32_t* kout, int* iout, int n, int shift,
                             const uint32_t* hist, int nblk) {
  __shared__ uint32_t offs[256];
  __shared__ uint32_t wc[RS_THREADS / 32][256];
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  offs[t] = hist[t * nblk + blockIdx.x];
  const unsigned lt = (1u << lane) - 1u;
  int base = blockIdx.x * RS_TILE;
  for (int r = 0; r < RS_ROUNDS; ++r) {
#pragma unroll
    for (int w = 0; w < RS_THREADS / 32; ++w) wc[w][t] = 0;
    __syncthreads();
    int idx = base + r * RS_THREADS + t;
    bool valid = idx < n;
    uint32_t key = valid ? kin[idx] : 0u;
    int id = valid ? iin[idx] : 0;
    int digit = valid ? (int)((key >> shift) & 255u) : 256;
    unsigned peers = __match_any_sync(0xffffffffu, digit);
    int rank = __popc(peers & lt);
    if (valid && rank == 0) wc[warp][digit] = __popc(peers);
    __syncthreads();
    uint32_t run = 0;
#pragma unroll
    for (int w = 0; w < RS_THREADS / 32; ++w) { uint32_t c = wc[w][t]; wc[w][t] = run; run += c; }
    __syncthreads();
    if (valid) {
      uint32_t dst = offs[digit] + wc[warp][digit] + rank;
      kout[dst] = key;
      iout[dst] = id;
    }
    __syncthreads();
    offs[t] += run;
    __syncthreads();
  }
}

// ---- Karras hierarchy
__device__ __forceinline__ int delta(const uint32_t* k, int n, int i, int j) {
  if (j < 0 || j >= n) return -1;
  uint32_t a = k[i], b = k[j];
  return a != b ? __clz(a ^ b) : 32 + __clz((uint32_t)i ^ (uint32_t)j);
}

__global__ void k_hierarchy(const uint32_t* keys, int n, float4* nodes, int* parent) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n - 1) return;
  int dir = (delta(keys, n, i, i + 1) - delta(keys, n, i, i - 1)) >= 0 ? 1 : -1;
  int dmin = delta(keys, n, i, i - dir);
  int lmax = 2;
  while (delta(keys, n, i, i + lmax * dir) > dmin) lmax <<= 1;
  int l = 0;
  for (int t = lmax >> 1; t >= 1; t >>= 1)
    if (delta(keys, n, i, i + (l + t) * dir) > dmin) l += t;
  int j = i + l * dir;
  int dnode = delta(keys, n, i, j);
  int s = 0, t = l;
  do {
    t = (t + 1) >> 1;
    if (delta(keys, n, i, i + (s + t) * dir) > dnode) s += t;
  } while (t > 1);
  int g = i + s * dir + min(dir, 0);
  int left = (min(i, j) == g) ? ~g : g;
  int right = (max(i, j) == g + 1) ? ~(g + 1) : g + 1;
  nodes[4 * i + 3] = make_float4(__int_as_float(left), __int_as_float(right), 0.0f, 0.0f);
  if (left < 0) parent[(n - 1) + ~left] = i; else parent[left] = i;
  if (right < 0) parent[(n - 1) + ~right] = i; else parent[right] = i;
  if (i == 0) parent[0] = -1;
}

// ---- leaf records and bottom-up boxes
__global__ void k_boxes(const float* V, const int* F, const int* ids, int n, float4* tri, float4* nodes,
                        const int* parent, int* flags, int* err) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int f = ids[i];
  int a = F[3 * f], b = F[3 * f + 1], c = F[3 * f + 2];
  float3 p0 = mk3(V[3 * a], V[3 * a + 1], V[3 * a + 2]);
  float3 p1 = mk3(V[3 * b], V[3 * b + 1], V[3 * b + 2]);
  float3 p2 = mk3(V[3 * c], V[3 * c + 1], V[3 * c + 2]);
  tri[3 * i] = make_float4(p0.x, p0.y, p0.z, __int_as_float(f));
  tri[3 * i + 1] = make_float4(p1.x, p1.y, p1.z, 0.0f);
  tri[3 * i + 2] = make_float4(p2.x, p2.y, p2.z, 0.0f);
  if (n == 1) return;
  float3 lo = mk3(fminf(fminf(p0.x, p1.x), p2.x), fminf(fminf(p0.y, p1.y), p2.y), fminf(fminf(p0.z, p1.z), p2.z));
  float3 hi = mk3(fmaxf(fmaxf(p0.x, p1.x), p2.x), fmaxf(fmaxf(p0.y, p1.y), p2.y), fmaxf(fmaxf(p0.z, p1.z), p2.z));
  int child = ~i;
  int node = parent[(n - 1) + i];
  for (int depth = 0; node >= 0; ++depth) {
    if (depth > 256) { atomicOr(err, 2); return; }  // deeper than any tree built here: malformed
    float4* np = nodes + 4 * node;
    int cl = __float_as_int(np[3].x);
    if (cl == child) {
      np[0] = make_float4(lo.x, hi.x, lo.y, hi.y);
      np[1].x = lo.z; np[1].y = hi.z;
    } else {
      np[1].z = lo.x; np[1].w = hi.x;
      np[2] = make_float4(lo.y, hi.y, lo.z, hi.z);
    }
    __threadfence();
    if (atomicAdd(&flags[node], 1) == 0) return;  // the sibling's thread finishes this node
    __threadfence();
    float4 n0 = __ldcg(np), n1 = __ldcg(np + 1), n2 = __ldcg(np + 2);
    lo = mk3(fminf(n0.x, n1.z), fminf(n0.z, n2.x), fminf(n1.x, n2.z));
    hi = mk3(fmaxf(n0.y, n1.w), fmaxf(n0.w, n2.y), fmaxf(n1.y, n2.w));
    child = node;
    node = parent[node];
  }
}

cudaError_t boxes(st_scene* s, cudaStream_t stream) {
  int n = s->nf;
  if (n > 1) {
    cudaError_t e = cudaMemsetAsync(s->flags, 0, sizeof(int) * (n - 1), stream);
    if (e != cudaSuccess) return e;
  }
  k_boxes<<<(n + 255) / 256, 256, 0, stream>>>(s->verts, s->faces, s->ids, n, s->tri, s->nodes, s->parent, s->flags,
                                                s->d_err);
  return cudaGetLastError();
}

}  // namespace

// ---- PLOC: Meister and Bittner, "Parallel Locally-Ordered Clustering for
// Bounding Volume Hierarchy Construction" (IEEE TVCG 2018). The leaves in
// Morton order are the initial clusters; every round each cluster finds, among
// the PLOC_R clusters on either side of it in the current order, the one whose
// merged box has the least surface area; mutual nearest neighbours merge into a
// new internal node that takes the lower position, and the array is compacted
// in order. Ties compare (area, lower index, higher index), a total order on
// pairs, so the closest pair of a round is always mutual and every round
// merges. Nodes are numbered downward from n - 2, so the last merge is the
// root, node 0; the result has the Karras layout (child links, parent array)
// that the bottom-up boxes, the refit and the 4-wide collapse read.
constexpr int PLOC_R = 16;
constexpr int PLOC_BLOCK = 256;
constexpr int SCAN2_BLOCK = 1024;

__global__ void k_ploc_init(const float* V, const int* F, const int* ids, int n, int* cid, float4* lo, float4* hi) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int f = ids[i];
  float3 p0 = mk3(V[3 * F[3 * f]], V[3 * F[3 * f] + 1], V[3 * F[3 * f] + 2]);
  float3 p1 = mk3(V[3 * F[3 * f + 1]], V[3 * F[3 * f + 1] + 1], V[3 * F[3 * f + 1] + 2]);
  float3 p2 = mk3(V[3 * F[3 * f + 2]], V[3 * F[3 * f + 2] + 1], V[3 * F[3 * f + 2] + 2]);
  lo[i] = make_float4(fminf(fminf(p0.x, p1.x), p2.x), fminf(fminf(p0.y, p1.y), p2.y), fminf(fminf(p0.z, p1.z), p2.z), 0.0f);
  hi[i] = make_float4(fmaxf(fmaxf(p0.x, p1.x), p2.x), fmaxf(fmaxf(p0.y, p1.y), p2.y), fmaxf(fmaxf(p0.z, p1.z), p2.z), 0.0f);
  cid[i] = ~i;
}

__device__ __forceinline__ float merged_area(float4 al, float4 ah, float4 bl, float4 bh) {
  float dx = fmaxf(ah.x, bh.x) - fminf(al.x, bl.x);
  float dy = fmaxf(ah.y, bh.y) - fminf(al.y, bl.y);
  float dz = fmaxf(ah.z, bh.z) - fminf(al.z, bl.z);
  return dx * dy + dy * dz + dz * dx;
}

__global__ void __launch_bounds__(PLOC_BLOCK) k_ploc_nn(const float4* lo, const float4* hi, int c, int* nn) {
  __shared__ float4 slo[PLOC_BLOCK + 2 * PLOC_R], shi[PLOC_BLOCK + 2 * PLOC_R];
  const int b0 = blockIdx.x * PLOC_BLOCK;
  for (int k = threadIdx.x; k < PLOC_BLOCK + 2 * PLOC_R; k += PLOC_BLOCK) {
    int g = b0 - PLOC_R + k;
    if (g >= 0 && g < c) {
      slo[k] = lo[g];
      shi[k] = hi[g];
    }
  }
  __syncthreads();
  int i = b0 + threadIdx.x;
  if (i >= c) return;
  float4 al = slo[threadIdx.x + PLOC_R], ah = shi[threadIdx.x + PLOC_R];
  float best = __int_as_float(0x7f800000);
  int bj = -1;
  // ascending j with a strict test keeps the least (area, lower index, higher index)
  for (int d = -PLOC_R; d <= PLOC_R; ++d) {
    int j = i + d;
    if (d == 0 || j < 0 || j >= c) continue;
    float a = merged_area(al, ah, slo[threadIdx.x + PLOC_R + d], shi[threadIdx.x + PLOC_R + d]);
    if (a < best) {
      best = a;
      bj = j;
    }
  }
  nn[i] = bj;
}

// (merges, survivors) flags of cluster i: i merges (as the lower of a mutual
// pair) or survives alone; the higher of a mutual pair disappears.
__device__ __forceinline__ int2 ploc_flags(const int* nn, int i) {
  int j = nn[i];
  bool mutual = j >= 0 && nn[j] == i;
  return make_int2(mutual && i < j ? 1 : 0, mutual && j < i ? 0 : 1);
}

__device__ __forceinline__ int2 add2(int2 a, int2 b) { return make_int2(a.x + b.x, a.y + b.y); }

__device__ __forceinline__ int2 block_scan2(int2 v, int2* sh, int2& total) {
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int2 x = v;
  for (int o = 1; o < 32; o <<= 1) {
    int2 y = make_int2(__shfl_up_sync(0xffffffffu, x.x, o), __shfl_up_sync(0xffffffffu, x.y, o));
    if (lane >= o) x = add2(x, y);
  }
  if (lane == 31) sh[w] = x;
  __syncthreads();
  if (w == 0) {
    int nw = blockDim.x >> 5;
    int2 t = lane < nw ? sh[lane] : make_int2(0, 0);
    for (int o = 1; o < 32; o <<= 1) {
      int2 y = make_int2(__shfl_up_sync(0xffffffffu, t.x, o), __shfl_up_sync(0xffffffffu, t.y, o));
      if (lane >= o) t = add2(t, y);
    }
    if (lane < nw) sh[lane] = t;
  }
  __syncthreads();
  int2 before = w > 0 ? sh[w - 1] : make_int2(0, 0);
  total = sh[(blockDim.x >> 5) - 1];
  return make_int2(before.x + x.x - v.x, before.y + x.y - v.y);   // exclusive
}

__global__ void __launch_bounds__(SCAN2_BLOCK) k_ploc_scan(const int* nn, int c, int2* scan, int2* part) {
  __shared__ int2 sh[32];
  int i = blockIdx.x * SCAN2_BLOCK + threadIdx.x;
  int2 v = i < c ? ploc_flags(nn, i) : make_int2(0, 0);
  int2 tot;
  int2 ex = block_scan2(v, sh, tot);
  if (i < c) scan[i] = ex;
  if (threadIdx.x == 0) part[blockIdx.x] = tot;
}

// exclusive scan of the block totals, in place; part[nb] = the grand total
__global__ void __launch_bounds__(SCAN2_BLOCK) k_ploc_parts(int2* part, int nb) {
  __shared__ int2 sh[32];
  int2 carry = make_int2(0, 0);
  for (int b = 0; b < nb; b += SCAN2_BLOCK) {
    int i = b + threadIdx.x;
    int2 v = i < nb ? part[i] : make_int2(0, 0);
    int2 tot;
    int2 ex = block_scan2(v, sh, tot);
    __syncthreads();
    if (i < nb) part[i] = add2(ex, carry);
    carry = add2(carry, tot);
    __syncthreads();
  }
  if (threadIdx.x == 0) part[nb] = carry;
}

__global__ void __launch_bounds__(SCAN2_BLOCK) k_ploc_merge(const int* nn, int c, const int2* scan, const int2* part,
                                                           int next, int n, const int* cid, const float4* lo,
                                                           const float4* hi, int* cid2, float4* lo2, float4* hi2,
                                                           float4* nodes, int* parent) {
  int i = blockIdx.x * SCAN2_BLOCK + threadIdx.x;
  if (i >= c) return;
  int2 f = ploc_flags(nn, i);
  int2 pos = add2(scan[i], part[blockIdx.x]);
  if (f.x) {
    int j = nn[i];
    int k = next - 1 - pos.x;
    int a = cid[i], b = cid[j];
    nodes[4 * k + 3] = make_float4(__int_as_float(a), __int_as_float(b), 0.0f, 0.0f);
    if (a >= 0) parent[a] = k; else parent[(n - 1) + ~a] = k;
    if (b >= 0) parent[b] = k; else parent[(n - 1) + ~b] = k;
    float4 al = lo[i], ah = hi[i], bl = lo[j], bh = hi[j];
    cid2[pos.y] = k;
    lo2[pos.y] = make_float4(fminf(al.x, bl.x), fminf(al.y, bl.y), fminf(al.z, bl.z), 0.0f);
    hi2[pos.y] = make_float4(fmaxf(ah.x, bh.x), fmaxf(ah.y, bh.y), fmaxf(ah.z, bh.z), 0.0f);
  } else if (f.y) {
    cid2[pos.y] = cid[i];
    lo2[pos.y] = lo[i];
    hi2[pos.y] = hi[i];
  }
}

namespace {
cudaError_t morton_order(st_scene* s, cudaStream_t stream) {
  int n = s->nf;
  k_init_bounds<<<1, 32, 0, stream>>>(s->bounds);
  int g = min((n + 255) / 256, 4 * max(s->sm_count, 1));
  k_centroid_bounds<<<g, 256, 0, stream>>>(s->verts, s->faces, n, s->bounds);
  k_morton<<<(n + 255) / 256, 256, 0, stream>>>(s->verts, s->faces, n, s->bounds, s->keys, s->ids);
  uint32_t *ka = s->keys, *kb = s->keys2;
  int *ia = s->ids, *ib = s->ids2;
  int nblk = s->sort_blocks;
  for (int shift = 0; shift < 32; shift += 8) {
    k_rs_hist<<<nblk, RS_THREADS, 0, stream>>>(ka, n, shift, s->hist, nblk);
    k_rs_scan<<<1, 1024, 0, stream>>>(s->hist, 256 * nblk);
    k_rs_scatter<<<nblk, RS_THREADS, 0, stream>>>(ka, ia, kb, ib, n, shift, s->hist, nblk);
    std::swap(ka, kb);
    std::swap(ia, ib);
  }
  // four passes: the sorted data is back in the primary buffers
  return cudaGetLastError();
}
}  // namespace

cudaError_t bvh_build(st_scene* s, cudaStream_t stream) {
  int n = s->nf;
  cudaError_t e = morton_order(s, stream);
  if (e != cudaSuccess) return e;
  if (n > 1) k_hierarchy<<<(n - 1 + 255) / 256, 256, 0, stream>>>(s->keys, n, s->nodes, s->parent);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return boxes(s, stream);
}

cudaError_t bvh_build_ploc(st_scene* s, cudaStream_t stream) {
  int n = s->nf;
  cudaError_t e = morton_order(s, stream);
  if (e != cudaSuccess || n < 2) return e != cudaSuccess ? e : boxes(s, stream);
  // scratch for the rounds: two cluster arrays (box, id), scans, neighbours
  int nb = (n + SCAN2_BLOCK - 1) / SCAN2_BLOCK;
  size_t bytes = 4 * (size_t)n * sizeof(float4) + (size_t)n * sizeof(int2) + (size_t)(nb + 1) * sizeof(int2) +
                 3 * (size_t)n * sizeof(int);
  char* buf = nullptr;
  e = cudaMalloc((void**)&buf, bytes);
  if (e != cudaSuccess) return e;
  float4* lo[2] = {(float4*)buf, (float4*)buf + n};
  float4* hi[2] = {(float4*)buf + 2 * (size_t)n, (float4*)buf + 3 * (size_t)n};
  int2* scan = (int2*)((float4*)buf + 4 * (size_t)n);
  int2* part = scan + n;
  int* cid[2] = {(int*)(part + nb + 1), (int*)(part + nb + 1) + n};
  int* nn = cid[1] + n;
  k_ploc_init<<<(n + 255) / 256, 256, 0, stream>>>(s->verts, s->faces, s->ids, n, cid[0], lo[0], hi[0]);
  int c = n, next = n - 1, cur = 0;
  int2 tot = make_int2(0, 0);
  for (int round = 0; c > 1 && e == cudaSuccess; ++round) {
    if (round > 4 * n) { e = cudaErrorIllegalState; break; }
    int g = (c + PLOC_BLOCK - 1) / PLOC_BLOCK, gs = (c + SCAN2_BLOCK - 1) / SCAN2_BLOCK;
    k_ploc_nn<<<g, PLOC_BLOCK, 0, stream>>>(lo[cur], hi[cur], c, nn);
    k_ploc_scan<<<gs, SCAN2_BLOCK, 0, stream>>>(nn, c, scan, part);
    k_ploc_parts<<<1, SCAN2_BLOCK, 0, stream>>>(part, gs);
    k_ploc_merge<<<gs, SCAN2_BLOCK, 0, stream>>>(nn, c, scan, part, next, n, cid[cur], lo[cur], hi[cur], cid[cur ^ 1],
                                                 lo[cur ^ 1], hi[cur ^ 1], s->nodes, s->parent);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(&tot, part + gs, sizeof(int2), cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) break;
    // a round without a merge means non-finite boxes
    if (tot.x <= 0 || tot.y != c - tot.x) { e = cudaErrorIllegalState; break; }
    next -= tot.x;
    c = tot.y;
    cur ^= 1;
  }
  if (e == cudaSuccess && next != 0) e = cudaErrorIllegalState;
  if (e == cudaSuccess) e = cudaMemsetAsync(s->parent, 0xff, sizeof(int), stream);   // the root has no parent
  if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
  cudaFree(buf);
  if (e != cudaSuccess) return e;
  return boxes(s, stream);
}

// ---- 4-wide collapse: each 4-wide node takes a binary node's children and
// repeatedly opens the internal child of largest surface area until it holds
// four children (or only leaves); the opened-up children become 4-wide nodes.
__device__ __forceinline__ float binary_area(const float4* nodes, int c) {
  const float4* np = nodes + 4 * c;
  float4 n0 = np[0], n1 = np[1], n2 = np[2];
  float dx = fmaxf(n0.y, n1.w) - fminf(n0.x, n1.z);
  float dy = fmaxf(n0.w, n2.y) - fminf(n0.z, n2.x);
  float dz = fmaxf(n1.y, n2.w) - fminf(n1.x, n2.z);
  return dx * dy + dy * dz + dz * dx;
}

constexpr int EMPTY4 = (int)0x80000000;

__global__ void k_collapse(const float4* nodes, const int* qin, int nin, int* qout, int* counters, int* src4,
                           float4* nodes4) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nin) return;
  int b = qin[2 * k], id = qin[2 * k + 1];
  float4 n3 = nodes[4 * b + 3];
  int slot[4] = {__float_as_int(n3.x), __float_as_int(n3.y), EMPTY4, EMPTY4};
  int n = 2;
  while (n < 4) {
    int best = -1;
    float ba = -1.0f;
    for (int j = 0; j < n; ++j)
      if (slot[j] >= 0) {
        float a = binary_area(nodes, slot[j]);
        if (a > ba) { ba = a; best = j; }
      }
    if (best < 0) break;
    float4 c3 = nodes[4 * slot[best] + 3];
    slot[best] = __float_as_int(c3.x);
    slot[n++] = __float_as_int(c3.y);
  }
  int child[4];
  for (int j = 0; j < 4; ++j) {
    int sj = slot[j];
    child[j] = sj;
    if (sj >= 0) {
      int nid = atomicAdd(&counters[0], 1);
      int qi = atomicAdd(&counters[1], 1);
      qout[2 * qi] = sj;
      qout[2 * qi + 1] = nid;
      child[j] = nid;
    }
    src4[4 * id + j] = sj;
  }
  nodes4[7 * id + 6] = make_float4(__int_as_float(child[0]), __int_as_float(child[1]), __int_as_float(child[2]),
                                   __int_as_float(child[3]));
}

// child boxes of every 4-wide node from the binary boxes / leaf triangles
__global__ void k_refit4(const float4* nodes, const float4* tri, const int* src4, int n4, float4* nodes4) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n4) return;
  float lo[3][4], hi[3][4];
  for (int j = 0; j < 4; ++j) {
    int sj = src4[4 * k + j];
    float3 a = mk3(1e30f, 1e30f, 1e30f), b = mk3(-1e30f, -1e30f, -1e30f);
    if (sj != EMPTY4 && sj < 0) {
      int li = ~sj;
      float3 p0 = xyz(tri[3 * li]), p1 = xyz(tri[3 * li + 1]), p2 = xyz(tri[3 * li + 2]);
      a = mk3(fminf(fminf(p0.x, p1.x), p2.x), fminf(fminf(p0.y, p1.y), p2.y), fminf(fminf(p0.z, p1.z), p2.z));
      b = mk3(fmaxf(fmaxf(p0.x, p1.x), p2.x), fmaxf(fmaxf(p0.y, p1.y), p2.y), fmaxf(fmaxf(p0.z, p1.z), p2.z));
    } else if (sj >= 0) {
      const float4* np = nodes + 4 * sj;
      float4 n0 = np[0], n1 = np[1], n2 = np[2];
      a = mk3(fminf(n0.x, n1.z), fminf(n0.z, n2.x), fminf(n1.x, n2.z));
      b = mk3(fmaxf(n0.y, n1.w), fmaxf(n0.w, n2.y), fmaxf(n1.y, n2.w));
    }
    lo[0][j] = a.x; lo[1][j] = a.y; lo[2][j] = a.z;
    hi[0][j] = b.x; hi[1][j] = b.y; hi[2][j] = b.z;
  }
  float4* o = nodes4 + 7 * k;
  for (int ax = 0; ax < 3; ++ax) {
    o[2 * ax] = make_float4(lo[ax][0], lo[ax][1], lo[ax][2], lo[ax][3]);
    o[2 * ax + 1] = make_float4(hi[ax][0], hi[ax][1], hi[ax][2], hi[ax][3]);
  }
}

cudaError_t refit4(st_scene* s, cudaStream_t stream) {
  if (!s->nodes4 || s->n4 <= 0) return cudaSuccess;
  k_refit4<<<(s->n4 + 127) / 128, 128, 0, stream>>>(s->nodes, s->tri, s->src4, s->n4, s->nodes4);
  return cudaGetLastError();
}

cudaError_t bvh_refit(st_scene* s, cudaStream_t stream) {
  cudaError_t e = boxes(s, stream);
  return e != cudaSuccess ? e : refit4(s, stream);
}

cudaError_t bvh_collapse(st_scene* s, cudaStream_t stream) {
  int n = s->nf;
  s->n4 = 0;
  if (n < 2) return cudaSuccess;
  int init[2] = {0, 0};   // binary root -> 4-wide node 0
  int cnt[2] = {1, 0};
  int* qa = s->q4;
  int* qb = s->q4 + 2 * (size_t)n;
  cudaError_t e = cudaMemcpyAsync(qa, init, sizeof(init), cudaMemcpyHostToDevice, stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(s->c4, cnt, sizeof(cnt), cudaMemcpyHostToDevice, stream);
  int nin = 1;
  for (int level = 0; nin > 0 && e == cudaSuccess; ++level) {
    if (level > 64) return cudaErrorIllegalState;  // deeper than any tree built here: malformed
    e = cudaMemsetAsync(s->c4 + 1, 0, sizeof(int), stream);
    if (e != cudaSuccess) break;
    k_collapse<<<(nin + 127) / 128, 128, 0, stream>>>(s->nodes, qa, nin, qb, s->c4, s->src4, s->nodes4);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(cnt, s->c4, sizeof(cnt), cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    nin = cnt[1];
    std::swap(qa, qb);
  }
  if (e != cudaSuccess) return e;
  s->n4 = cnt[0];
  return refit4(s, stream);
}

int sort_blocks_for(int n) { return (n + RS_TILE - 1) / RS_TILE; }

// ---- mesh statistics for back-face culling of the primary-visibility bins
__global__ void k_mesh_stat_init(MeshStat* m) {
  m->vol6 = 0.0;
  m->winding = 0;
  for (int k = 0; k < 3; ++k) {
    m->lo[k] = 0x7fffffff;
    m->hi[k] = (int)0x80000000;
  }
}

__global__ void k_mesh_stat(const float* V, int nv, const int* F, int nf, MeshStat* m) {
  __shared__ double sv[8];
  double v = 0.0;
  for (int f = blockIdx.x * blockDim.x + threadIdx.x; f < nf; f += gridDim.x * blockDim.x) {
    const int* fi = F + 3 * f;
    double a[3], b[3], c[3];
    for (int k = 0; k < 3; ++k) {
      a[k] = V[3 * fi[0] + k]; b[k] = V[3 * fi[1] + k]; c[k] = V[3 * fi[2] + k];
    }
    v += a[0] * (b[1] * c[2] - b[2] * c[1]) - a[1] * (b[0] * c[2] - b[2] * c[0]) + a[2] * (b[0] * c[1] - b[1] * c[0]);
  }
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) sv[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sv[w];
    atomicAdd(&m->vol6, t);
  }
  int lo[3] = {0x7fffffff, 0x7fffffff, 0x7fffffff}, hi[3] = {(int)0x80000000, (int)0x80000000, (int)0x80000000};
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nv; i += gridDim.x * blockDim.x)
    for (int k = 0; k < 3; ++k) {
      int q = ordered(V[3 * i + k]);
      lo[k] = min(lo[k], q);
      hi[k] = max(hi[k], q);
    }
  for (int k = 0; k < 3; ++k) {
    for (int o = 16; o > 0; o >>= 1) {
      lo[k] = min(lo[k], __shfl_xor_sync(0xffffffffu, lo[k], o));
      hi[k] = max(hi[k], __shfl_xor_sync(0xffffffffu, hi[k], o));
    }
    if ((threadIdx.x & 31) == 0) {
      atomicMin(&m->lo[k], lo[k]);
      atomicMax(&m->hi[k], hi[k]);
    }
  }
}

// the winding's sign only where the volume is clearly nonzero (a thousandth of the bounding box's)
__global__ void k_mesh_stat_final(MeshStat* m) {
  double d[3];
  for (int k = 0; k < 3; ++k) d[k] = (double)unordered(m->hi[k]) - (double)unordered(m->lo[k]);
  double box6 = 6.0 * d[0] * d[1] * d[2];
  m->winding = fabs(m->vol6) > 1e-3 * box6 ? (m->vol6 > 0.0 ? 1 : -1) : 0;
}

// Vertex normals for interpolated shading: M_v = the sum of (v1 - v0) x (v2 - v0)
// over the faces around v in face order (one thread per vertex, so the sum's
// order is fixed), stored as (M_v / |M_v|, |M_v|).
__global__ void k_vertex_normals(const float* V, const int* F, const int* vf_start, const int* vf_list, int nv,
                                 float4* out) {
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < nv; v += gridDim.x * blockDim.x) {
    float3 M = mk3(0, 0, 0);
    for (int k = vf_start[v]; k < vf_start[v + 1]; ++k) {
      int f = vf_list[k];
      auto vx = [&](int i) { return mk3(V[3 * i], V[3 * i + 1], V[3 * i + 2]); };
      float3 a = vx(F[3 * f]), b = vx(F[3 * f + 1]), c = vx(F[3 * f + 2]);
      M += cross3(b - a, c - a);
    }
    float l = len3(M);
    out[v] = make_float4(M.x / l, M.y / l, M.z / l, l);
  }
}

cudaError_t mesh_stat(st_scene* s, cudaStream_t stream) {
  if (s->smooth && s->vnrm) {
    int gv = std::min((s->nv + 255) / 256, 4 * std::max(s->sm_count, 1));
    k_vertex_normals<<<gv, 256, 0, stream>>>(s->verts, s->faces, s->vf_start, s->vf_list, s->nv, s->vnrm);
  }
  if (!s->mstat) return cudaSuccess;
  k_mesh_stat_init<<<1, 1, 0, stream>>>(s->mstat);
  int g = std::min((std::max(s->nf, s->nv) + 255) / 256, 4 * std::max(s->sm_count, 1));
  k_mesh_stat<<<g, 256, 0, stream>>>(s->verts, s->nv, s->faces, s->nf, s->mstat);
  k_mesh_stat_final<<<1, 1, 0, stream>>>(s->mstat);
  return cudaGetLastError();
}

}  // namespace st
