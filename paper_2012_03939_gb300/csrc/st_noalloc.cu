// Allocation-free LBVH build (st_build_bvh_noalloc).
//
// Some callers cannot allocate device memory at the moment they need a BVH:
// code running under an allocator that is already at its budget, inside a
// framework that forbids allocation on its hot path, or an embedding that owns
// every buffer itself. This entry point runs the same build as
// st_scene_create (Morton codes, radix sort, Karras hierarchy, bottom-up
// boxes) but takes its scratch -- sort keys and ids, histograms, parent links,
// visit counters -- from one file-scope device array of fixed size instead of
// cudaMalloc. The caller passes the mesh and the output buffers.
#include <mutex>

#include "st_internal.h"

namespace st {
namespace {

constexpr int NA_MAX_FACES = 1 << 16;                  // largest mesh this entry point accepts
constexpr int NA_SORT_BLOCKS = (NA_MAX_FACES + 4095) / 4096;
// scratch layout, in 4-byte words
constexpr size_t NA_KEYS = 0;
constexpr size_t NA_KEYS2 = NA_KEYS + NA_MAX_FACES;
constexpr size_t NA_IDS = NA_KEYS2 + NA_MAX_FACES;
constexpr size_t NA_IDS2 = NA_IDS + NA_MAX_FACES;
constexpr size_t NA_PARENT = NA_IDS2 + NA_MAX_FACES;   // 2 * F words
constexpr size_t NA_FLAGS = NA_PARENT + 2 * (size_t)NA_MAX_FACES;
constexpr size_t NA_HIST = NA_FLAGS + NA_MAX_FACES;    // 256 * sort blocks
constexpr size_t NA_BOUNDS = NA_HIST + 256 * (size_t)NA_SORT_BLOCKS;
constexpr size_t NA_ERR = NA_BOUNDS + 8;
constexpr size_t NA_WORDS = NA_ERR + 8;                // about 1.8 MiB

// Every device that loads the library holds this array until the process exits.
static __device__ __align__(256) uint32_t g_noalloc_scratch[NA_WORDS];

constexpr int NA_MAX_DEVICES = 64;
std::mutex g_na_mutex;
uint32_t* g_na_ptr[NA_MAX_DEVICES] = {};

// Device address of the scratch array on the current device, looked up once
// per device (host code only sees a stand-in for the symbol, not its address).
cudaError_t scratch_address(uint32_t** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= NA_MAX_DEVICES) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_na_mutex);
  if (!g_na_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_na_ptr[dev] = static_cast<uint32_t*>(p);
  }
  *out = g_na_ptr[dev];
  return cudaSuccess;
}

__global__ void k_na_check_faces(const int* F, int nf, int nv, int* err) {
  int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= nf) return;
  int a = F[3 * f], b = F[3 * f + 1], c = F[3 * f + 2];
  if (a < 0 || b < 0 || c < 0 || a >= nv || b >= nv || c >= nv || a == b || b == c || a == c) atomicOr(err, 1);
}

}  // namespace
}  // namespace st

using namespace st;

extern "C" st_status st_build_bvh_noalloc(const float* vertices, const int* faces, int n_vertices, int n_faces,
                                          float* nodes, float* tris, int* leaf_faces, void* stream) {
  if (n_faces <= 0 || n_vertices <= 0 || !vertices || !faces || !tris || !leaf_faces || (n_faces > 1 && !nodes)) {
    set_error("st_build_bvh_noalloc: missing argument");
    return ST_ERR_INVALID_ARG;
  }
  if (n_faces > NA_MAX_FACES) {
    set_error("st_build_bvh_noalloc: " + std::to_string(n_faces) + " faces exceed the fixed scratch limit of " +
              std::to_string(NA_MAX_FACES));
    return ST_ERR_UNSUPPORTED;
  }
  if (((uintptr_t)tris & 15) || ((uintptr_t)nodes & 15)) {
    set_error("st_build_bvh_noalloc: nodes and tris must be 16-byte aligned");
    return ST_ERR_INVALID_ARG;
  }
  cudaStream_t st = (cudaStream_t)stream;
  uint32_t* w = nullptr;
  cudaError_t e = scratch_address(&w);
  if (e != cudaSuccess) {
    set_error(std::string("st_build_bvh_noalloc: scratch lookup: ") + cudaGetErrorString(e));
    return ST_ERR_CUDA;
  }
  int* err = (int*)(w + NA_ERR);
  // the array keeps the previous call's contents: clear the error word here;
  // bounds, histograms and visit counters are reset by the build itself
  e = cudaMemsetAsync(err, 0, sizeof(int), st);
  if (e == cudaSuccess) {
    k_na_check_faces<<<(n_faces + 255) / 256, 256, 0, st>>>(faces, n_faces, n_vertices, err);
    e = cudaGetLastError();
  }
  int herr = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    set_error(std::string("st_build_bvh_noalloc: ") + cudaGetErrorString(e));
    return ST_ERR_CUDA;
  }
  if (herr) {
    set_error("st_build_bvh_noalloc: face index out of range or degenerate face");
    return ST_ERR_INVALID_ARG;
  }
  st_scene s;  // a view onto caller buffers and the static scratch; owns nothing
  cudaGetDevice(&s.device);
  cudaDeviceGetAttribute(&s.sm_count, cudaDevAttrMultiProcessorCount, s.device);
  s.nv = n_vertices;
  s.nf = n_faces;
  s.verts = const_cast<float*>(vertices);
  s.faces = const_cast<int*>(faces);
  s.tri = (float4*)tris;
  s.nodes = (float4*)nodes;
  s.keys = w + NA_KEYS;
  s.keys2 = w + NA_KEYS2;
  s.ids = (int*)(w + NA_IDS);
  s.ids2 = (int*)(w + NA_IDS2);
  s.parent = (int*)(w + NA_PARENT);
  s.flags = (int*)(w + NA_FLAGS);
  s.hist = w + NA_HIST;
  s.bounds = (int*)(w + NA_BOUNDS);
  s.d_err = err;
  s.sort_blocks = sort_blocks_for(n_faces);
  e = bvh_build(&s, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(leaf_faces, s.ids, sizeof(int) * n_faces, cudaMemcpyDeviceToDevice, st);
  // the bottom-up box pass latches an error bit in the same word when the tree it walks is malformed
  if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    set_error(std::string("st_build_bvh_noalloc: ") + cudaGetErrorString(e));
    return ST_ERR_CUDA;
  }
  if (herr) {
    set_error("st_build_bvh_noalloc: the build latched device error bits " + std::to_string(herr));
    return ST_ERR_DEVICE;
  }
  return ST_OK;
}
