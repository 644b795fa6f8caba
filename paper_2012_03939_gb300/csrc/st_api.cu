// C ABI of libst: scene lifetime, host-side preprocessing (edge list, FP64
// alias table), per-call planning of the job space, the wavefront chunk loop in
// its two launch modes (batched persistent + CUDA graph, or plain per-view),
// and statistics.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdlib>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "st_kernels.cuh"

namespace st {

// NVTX range for the lifetime of a scope: names the host-side enqueue of each
// call and wavefront stage for profilers (a captured graph replays as one range)
struct Range {
  explicit Range(const char* name) { nvtxRangePushA(name); }
  ~Range() { nvtxRangePop(); }
  Range(const Range&) = delete;
  Range& operator=(const Range&) = delete;
};

static thread_local std::string g_err;
void set_error(const std::string& msg) { g_err = msg; }

// Host-side fault injection (st_inject_fault): per site, the number of events
// to let pass before one fails (-1 = disarmed). The first query reads the
// ST_FAULT environment variable ("alloc:N" or "copy:N").
static std::atomic<int> g_fault[3] = {{-1}, {-1}, {-1}};

static void fault_from_env() {
  const char* v = std::getenv("ST_FAULT");
  if (!v) return;
  std::string s(v);
  size_t c = s.find(':');
  std::string site = s.substr(0, c);
  int n = c == std::string::npos ? 0 : std::atoi(s.c_str() + c + 1);
  if (site == "alloc") g_fault[ST_FAULT_ALLOC].store(n);
  else if (site == "copy") g_fault[ST_FAULT_COPY].store(n);
}

static void fault_init() {
  static const bool env_read = (fault_from_env(), true);
  (void)env_read;
}

bool fault_now(int site) {
  fault_init();
  int v = g_fault[site].load();
  while (v >= 0)
    if (g_fault[site].compare_exchange_weak(v, v - 1)) return v == 0;
  return false;
}

namespace {

constexpr int DEFAULT_CHUNK = 1 << 22;
// Faces per bin cell a view may hold, over the whole screen, before its cells are split further
constexpr double BIN_FACES_PER_CELL = 0.5;
// Segment bases and chunk sizes are multiples of 64: an edge segment is laid out
// in blocks of 64 jobs, the minus sides of 32 consecutive samples then their plus
// sides, so every warp traces one side along one edge (same behaviour per lane).
constexpr long long SEG_ALIGN = 64;

st_status fail(st_status s, const std::string& msg) {
  set_error(msg);
  return s;
}

st_status cuda_fail(cudaError_t e, const char* where) {
  return fail(ST_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define ST_CUDA(call)                                   \
  do {                                                  \
    cudaError_t e_ = (call);                            \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
  } while (0)

template <class T>
cudaError_t dalloc(T** p, size_t n, long long* acc = nullptr) {
  *p = nullptr;
  if (n == 0) return cudaSuccess;
  if (fault_now(ST_FAULT_ALLOC)) return cudaErrorMemoryAllocation;   // injected on the host, before CUDA
  if (acc) *acc += (long long)(n * sizeof(T));
  return cudaMalloc((void**)p, n * sizeof(T));
}

// Host<->device copies of scene, call and statistics data go through these, so
// an injected copy fault reaches every caller's error path.
cudaError_t copy_async(void* dst, const void* src, size_t bytes, cudaMemcpyKind kind, cudaStream_t st) {
  if (fault_now(ST_FAULT_COPY)) return cudaErrorInvalidValue;
  return cudaMemcpyAsync(dst, src, bytes, kind, st);
}

cudaError_t copy_sync(void* dst, const void* src, size_t bytes, cudaMemcpyKind kind) {
  if (fault_now(ST_FAULT_COPY)) return cudaErrorInvalidValue;
  return cudaMemcpy(dst, src, bytes, kind);
}

template <class T>
void dfree(T*& p) {
  if (p) cudaFree((void*)p);
  p = nullptr;
}

// Vose's alias method over texel weights lum * sin(theta at the row centre),
// built in double precision: small and large worklists are stacks seeded in
// index order; a small bin takes the top large bin as alias, which keeps
// (q_l + q_s) - 1 and moves to the small list once below one.
bool build_alias(const float* rgb, int w, int h, std::vector<float4>& tex, std::vector<float2>& tab) {
  const int N = w * h;
  std::vector<double> wt(N), q(N), prob(N, 1.0);
  std::vector<int> alias(N);
  double total = 0;
  const double PI = 3.14159265358979323846;
  for (int r = 0; r < h; ++r) {
    double s = std::sin(PI * (r + 0.5) / h);
    for (int c = 0; c < w; ++c) {
      const float* t = rgb + 3 * ((size_t)r * w + c);
      double l = 0.2126 * (double)t[0] + 0.7152 * (double)t[1] + 0.0722 * (double)t[2];
      wt[(size_t)r * w + c] = l * s;
    }
  }
  for (int i = 0; i < N; ++i) {
    if (!(wt[i] >= 0.0) || !std::isfinite(wt[i])) return false;
    total += wt[i];
  }
  if (!(total > 0.0)) return false;
  std::vector<int> small, large;
  for (int i = 0; i < N; ++i) {
    q[i] = (wt[i] * N) / total;
    alias[i] = i;
    (q[i] < 1.0 ? small : large).push_back(i);
  }
  while (!small.empty() && !large.empty()) {
    int a = small.back();
    small.pop_back();
    int b = large.back();
    prob[a] = q[a];
    alias[a] = b;
    q[b] = (q[b] + q[a]) - 1.0;
    if (q[b] < 1.0) {
      large.pop_back();
      small.push_back(b);
    }
  }
  for (int i : large) { prob[i] = 1.0; alias[i] = i; }
  for (int i : small) { prob[i] = 1.0; alias[i] = i; }
  tex.resize(N);
  tab.resize(N);
  for (int i = 0; i < N; ++i) {
    const float* t = rgb + 3 * (size_t)i;
    tex[i] = make_float4(t[0], t[1], t[2], (float)(wt[i] / total));
    float abits;
    std::memcpy(&abits, &alias[i], sizeof(float));
    tab[i] = make_float2((float)prob[i], abits);
  }
  return true;
}

// Undirected edges sorted by (min vertex, max vertex) with up to two faces.
void build_edges(const std::vector<int>& F, int nf, std::vector<int2>& ev, std::vector<int2>& ef) {
  std::vector<std::pair<unsigned long long, int>> e;
  e.reserve(3 * (size_t)nf);
  for (int f = 0; f < nf; ++f)
    for (int k = 0; k < 3; ++k) {
      unsigned a = (unsigned)F[3 * f + k], b = (unsigned)F[3 * f + (k + 1) % 3];
      unsigned lo = std::min(a, b), hi = std::max(a, b);
      e.push_back({((unsigned long long)lo << 32) | hi, f});
    }
  std::sort(e.begin(), e.end());
  ev.clear();
  ef.clear();
  for (size_t i = 0; i < e.size();) {
    size_t j = i;
    while (j < e.size() && e[j].first == e[i].first) ++j;
    ev.push_back(make_int2((int)(e[i].first >> 32), (int)(e[i].first & 0xffffffffu)));
    int second = j - i == 1 ? -1 : (j - i == 2 ? e[i + 1].second : -2);
    ef.push_back(make_int2(e[i].second, second));
    i = j;
  }
}

// True when the faces form one connected surface (across shared edges) in
// which every edge has exactly two faces that traverse it in opposite
// directions: a closed, consistently wound mesh. Seen from outside its bounds,
// such a surface is first hit on a face wound toward the eye (the outward side
// when the signed volume is positive), so the other faces can be left out of
// the primary-visibility bins.
bool closed_single_surface(const std::vector<int>& F, int nf, const std::vector<int2>& ef) {
  std::vector<unsigned long long> dir;
  dir.reserve(3 * (size_t)nf);
  for (int f = 0; f < nf; ++f)
    for (int k = 0; k < 3; ++k)
      dir.push_back(((unsigned long long)(unsigned)F[3 * f + k] << 32) | (unsigned)F[3 * f + (k + 1) % 3]);
  std::sort(dir.begin(), dir.end());
  for (size_t i = 0; i < dir.size(); ++i) {
    if (i > 0 && dir[i] == dir[i - 1]) return false;                      // an edge traversed twice the same way
    unsigned long long rev = (dir[i] << 32) | (dir[i] >> 32);
    if (!std::binary_search(dir.begin(), dir.end(), rev)) return false;   // a boundary edge
  }
  std::vector<int> up(nf);
  for (int f = 0; f < nf; ++f) up[f] = f;
  auto root = [&](int x) { while (up[x] != x) { up[x] = up[up[x]]; x = up[x]; } return x; };
  int comps = nf;
  for (const int2& e : ef) {
    if (e.y < 0) return false;
    int a = root(e.x), b = root(e.y);
    if (a != b) { up[a] = b; --comps; }
  }
  return comps == 1;
}

DevView make_view(const st_view& v, int spp) {
  double eye[3] = {v.eye[0], v.eye[1], v.eye[2]};
  double f[3] = {v.target[0] - eye[0], v.target[1] - eye[1], v.target[2] - eye[2]};
  double fl = std::sqrt(f[0] * f[0] + f[1] * f[1] + f[2] * f[2]);
  for (double& x : f) x /= fl;
  double up[3] = {v.up[0], v.up[1], v.up[2]};
  double r[3] = {f[1] * up[2] - f[2] * up[1], f[2] * up[0] - f[0] * up[2], f[0] * up[1] - f[1] * up[0]};
  double rl = std::sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
  for (double& x : r) x /= rl;
  double u[3] = {r[1] * f[2] - r[2] * f[1], r[2] * f[0] - r[0] * f[2], r[0] * f[1] - r[1] * f[0]};
  double th = std::tan((double)v.fov_y_deg * 3.14159265358979323846 / 360.0);
  DevView d;
  d.eye = mk3(v.eye[0], v.eye[1], v.eye[2]);
  d.fwd = mk3((float)f[0], (float)f[1], (float)f[2]);
  d.right = mk3((float)r[0], (float)r[1], (float)r[2]);
  d.up = mk3((float)u[0], (float)u[1], (float)u[2]);
  d.kx = (float)(th * v.width / v.height);
  d.ky = (float)th;
  d.W = v.width;
  d.H = v.height;
  d.spp = spp;
  d.off = (uint32_t)v.pixel_offset;
  d.pix_off = v.pixel_offset;
  d.nvl = v.n_lights;
  for (int j = 0; j < 4; ++j) d.vl[j] = make_float4(0, 0, 0, 0);
  for (int j = 0; j < v.n_lights && j < ST_MAX_VIEW_LIGHTS; ++j) {
    d.vl[2 * j] = make_float4(v.lights[j].pos[0], v.lights[j].pos[1], v.lights[j].pos[2], 0.0f);
    d.vl[2 * j + 1] = make_float4(v.lights[j].intensity[0], v.lights[j].intensity[1], v.lights[j].intensity[2], 0.0f);
  }
  return d;
}

bool view_ok(const st_view& v) {
  auto fin = [](const float* a, int n) {
    for (int i = 0; i < n; ++i)
      if (!std::isfinite(a[i])) return false;
    return true;
  };
  if (v.width <= 0 || v.height <= 0 || v.pixel_offset < 0 || v.spp < 0) return false;
  if (!fin(v.eye, 3) || !fin(v.target, 3) || !fin(v.up, 3) || !(v.fov_y_deg > 0 && v.fov_y_deg < 180)) return false;
  double f[3] = {v.target[0] - v.eye[0], v.target[1] - v.eye[1], v.target[2] - v.eye[2]};
  double c[3] = {f[1] * v.up[2] - f[2] * v.up[1], f[2] * v.up[0] - f[0] * v.up[2], f[0] * v.up[1] - f[1] * v.up[0]};
  return c[0] * c[0] + c[1] * c[1] + c[2] * c[2] > 0;
}

// ------------------------------------------------------------------ per-call plan
struct Plan {
  int kind = 0;  // 0 forward, 1 backward
  int B = 1;
  std::vector<DevView> views;
  std::vector<Seg> segs;
  std::vector<std::pair<long long, long long>> view_range;  // job range per view (per-view mode)
  long long total = 0;
  long long pixels = 0;       // sum of W*H: the call's pixel space (accumulation)
  long long cells = 0;        // sum of W*H*kb^2: the primary-visibility bin space
  bool interior = false, edges = false;
  bool sec = false;           // secondary-visibility edge samples at every camera-path vertex
  bool sec_tree = false;      // ... picked through the edge hierarchy
  bool shadow = false;        // point-light shadow-edge samples
  std::vector<int2> pairs;    // shadow edges: (view, light) of each candidate list
  bool sig = false;           // forward: path signatures
  int max_vl = 0;             // most point lights a view of the call adds to the scene's
  bool bins = false;          // build primary-visibility bins (worth it only for many primary rays)
  bool bins_reused = false;   // the previous build's lists serve this call (same views, same vertices)
  bool lbins = false;         // point-light shadow lists (scene lights, calls with many rays)
  bool lbins_reused = false;  // ... as the last build left them (no vertex update since)
  st_render_opts o{};
};

st_render_opts default_opts() {
  st_render_opts o;
  std::memset(&o, 0, sizeof(o));
  o.use_graph = 1;
  o.edge_mode = ST_EDGE_SILHOUETTE;
  return o;
}

void free_engine(Engine& e) {
  dfree(e.o); dfree(e.d); dfree(e.thr); dfree(e.rad); dfree(e.ctr); dfree(e.hit); dfree(e.origin);
  dfree(e.q0); dfree(e.q1); dfree(e.qs); dfree(e.sh_dir); dfree(e.sh_c);
  dfree(e.r0); dfree(e.r1); dfree(e.r2); dfree(e.r3); dfree(e.esc); dfree(e.nb); dfree(e.cnt); dfree(e.stat);
  dfree(e.sj); dfree(e.sje); dfree(e.pinj); dfree(e.sig); dfree(e.shr);
  e = Engine();
}

void drop_graphs(st_scene* s) {
  for (auto& g : s->graphs)
    if (g.exec) cudaGraphExecDestroy(g.exec);
  s->graphs.clear();
}

st_status grow_engine(st_scene* s, Engine& e, int Q, int B, int NS, bool records, bool sec, bool shadow) {
  if (e.Q >= Q && e.NS >= NS && (!records || (e.records && e.B >= B)) &&
      (!sec || e.sec_cap >= (long long)e.B * e.Q) && (!shadow || e.shadow))
    return ST_OK;
  // grow: keep the larger of old and new sizes so alternating calls do not thrash
  int nQ = std::max(Q, e.Q), nNS = std::max(NS, e.NS), nB = std::max(B, e.B);
  bool nrec = records || e.records;
  bool nsec = sec || e.sec_cap > 0;
  bool nshadow = shadow || e.shadow;
  cudaDeviceSynchronize();
  drop_graphs(s);
  free_engine(e);
  long long acc = 0;
  size_t q = (size_t)nQ;
  cudaError_t r = cudaSuccess;
  auto chk = [&](cudaError_t x) { if (x != cudaSuccess && r == cudaSuccess) r = x; };
  chk(dalloc(&e.o, q, &acc)); chk(dalloc(&e.d, q, &acc)); chk(dalloc(&e.thr, q, &acc)); chk(dalloc(&e.rad, q, &acc));
  chk(dalloc(&e.ctr, q, &acc)); chk(dalloc(&e.hit, q, &acc)); chk(dalloc(&e.origin, q, &acc));
  chk(dalloc(&e.q0, q, &acc)); chk(dalloc(&e.q1, q, &acc)); chk(dalloc(&e.qs, q, &acc));
  chk(dalloc(&e.sh_dir, q * std::max(nNS, 1), &acc)); chk(dalloc(&e.sh_c, q * std::max(nNS, 1), &acc));
  if (nrec) {
    chk(dalloc(&e.r0, q * nB, &acc)); chk(dalloc(&e.r1, q * (nB + 1), &acc)); chk(dalloc(&e.r2, q * nB, &acc));
    chk(dalloc(&e.r3, q * nB, &acc)); chk(dalloc(&e.esc, q, &acc)); chk(dalloc(&e.nb, q, &acc));
  }
  if (nsec) {
    chk(dalloc(&e.sj, 4 * q * nB, &acc)); chk(dalloc(&e.sje, q * nB, &acc)); chk(dalloc(&e.pinj, q * nB, &acc));
  }
  if (nshadow) chk(dalloc(&e.shr, 3 * q, &acc));
  chk(dalloc(&e.sig, q, &acc));
  chk(dalloc(&e.cnt, CNT_SIZE, &acc));
  chk(dalloc(&e.stat, STAT_SIZE, &acc));
  if (r != cudaSuccess) {
    free_engine(e);
    cudaGetLastError();
    return fail(ST_ERR_OOM, std::string("wavefront buffers: ") + cudaGetErrorString(r));
  }
  e.Q = nQ; e.B = nB; e.NS = nNS; e.records = nrec; e.bytes = acc;
  e.sec_cap = nsec ? (long long)nB * nQ : 0;
  e.shadow = nshadow;
  return ST_OK;
}

// The call's wavefront buffers: one engine, or all OVERLAP_ENGINES when consecutive
// chunks are to overlap on their streams (see enqueue_body).
st_status ensure_engine(st_scene* s, int Q, int B, int NS, bool records, bool sec, bool shadow, bool two) {
  st_status r = grow_engine(s, s->eng, Q, B, NS, records, sec, shadow);
  for (int k = 0; r == ST_OK && two && k < OVERLAP_ENGINES - 1; ++k)
    r = grow_engine(s, s->eng2[k], Q, B, NS, records, sec, shadow);
  return r;
}

st_status ensure_tables(st_scene* s, int n_views, int n_segs, bool edges) {
  int need = std::max(n_views, n_segs);
  if (need > s->view_cap) {
    cudaDeviceSynchronize();
    drop_graphs(s);
    dfree(s->d_views);
    dfree(s->d_segs);
    if (dalloc(&s->d_views, need) != cudaSuccess || dalloc(&s->d_segs, need) != cudaSuccess) {
      // leave no capacity behind a freed table: the next call allocates again
      dfree(s->d_views);
      dfree(s->d_segs);
      s->view_cap = 0;
      cudaGetLastError();
      return fail(ST_ERR_OOM, "view tables");
    }
    s->view_cap = need;
  }
  if (edges && n_views > s->edge_cap_views) {
    cudaDeviceSynchronize();
    drop_graphs(s);
    dfree(s->edge_flag);
    dfree(s->edge_cand);
    dfree(s->edge_ncand);
    size_t n = (size_t)n_views * std::max(s->n_edges, 1);
    if (dalloc(&s->edge_flag, n) != cudaSuccess || dalloc(&s->edge_cand, n) != cudaSuccess ||
        dalloc(&s->edge_ncand, (size_t)n_views) != cudaSuccess) {
      dfree(s->edge_flag);
      dfree(s->edge_cand);
      dfree(s->edge_ncand);
      s->edge_cap_views = 0;
      cudaGetLastError();
      return fail(ST_ERR_OOM, "edge tables");
    }
    s->edge_cap_views = n_views;
  }
  return ST_OK;
}

st_status ensure_bins(st_scene* s, const Plan& p) {
  long long P = p.cells;
  long long want = std::max<long long>(4 * P, 1 << 20);
  if (s->bin_total_host && *s->bin_total_host > s->bin_cap) want = std::max(want, 2LL * *s->bin_total_host);
  want = std::min<long long>(want, 0x7ffffff0LL);   // a clamped total (INT_MAX) always exceeds it
  bool grow = P > s->bin_pix_cap || (int)p.views.size() > s->bin_views_cap || want > s->bin_cap;
  if (!grow) return ST_OK;
  cudaDeviceSynchronize();
  drop_graphs(s);
  s->bins_valid = false;
  long long nP = std::max(P, s->bin_pix_cap), nC = std::max(want, s->bin_cap);
  int nV = std::max((int)p.views.size(), s->bin_views_cap);
  dfree(s->bin_start); dfree(s->bin_cur); dfree(s->bin_list); dfree(s->bin_ok); dfree(s->bin_part);
  long long nb = (nP + 4095) / 4096;
  if (dalloc(&s->bin_start, (size_t)nP + 1) != cudaSuccess || dalloc(&s->bin_cur, (size_t)nP) != cudaSuccess ||
      dalloc(&s->bin_list, (size_t)nC) != cudaSuccess || dalloc(&s->bin_ok, (size_t)nV) != cudaSuccess ||
      dalloc(&s->bin_part, (size_t)nb) != cudaSuccess) {
    dfree(s->bin_start); dfree(s->bin_cur); dfree(s->bin_list); dfree(s->bin_ok); dfree(s->bin_part);
    s->bin_pix_cap = 0; s->bin_cap = 0; s->bin_views_cap = 0;
    cudaGetLastError();
    return fail(ST_ERR_OOM, "primary-visibility bins");
  }
  if (!s->bin_total_host) cudaMallocHost((void**)&s->bin_total_host, sizeof(int));
  if (s->bin_total_host) *s->bin_total_host = 0;
  s->bin_pix_cap = nP; s->bin_cap = nC; s->bin_views_cap = nV;
  return ST_OK;
}

void free_light_bins(st_scene* s) {
  dfree(s->d_lviews); dfree(s->lbin_start); dfree(s->lbin_cur); dfree(s->lbin_list); dfree(s->lbin_ok);
  dfree(s->lbin_part);
  s->lbin_cells = 0;
  s->lbin_cap = 0;
}

// The point-light shadow lists, allocated by the first call that uses them: lbin_res^2 cells per scene light
// (lbin_res = 2 sqrt(F), in [16, 2048]: a closed mesh seen from a light outside it turns about F/2 faces toward
// the light, a few per ten cells of its disk); the list store grows when the last build's total (read back as
// for the primary-visibility bins) overflowed it.
st_status ensure_light_bins(st_scene* s) {
  if (s->lbin_res == 0) s->lbin_res = (int)std::min(2048.0, std::max(16.0, std::ceil(2.0 * std::sqrt((double)s->nf))));
  const long long R = s->lbin_res, P = (long long)s->nl * R * R;
  long long want = std::max<long long>(4 * P, 1 << 20);
  if (s->lbin_total_host && *s->lbin_total_host > s->lbin_cap) want = std::max(want, 2LL * *s->lbin_total_host);
  want = std::min<long long>(want, 0x7ffffff0LL);
  if (s->lbin_start && want <= s->lbin_cap) return ST_OK;
  cudaDeviceSynchronize();
  drop_graphs(s);
  s->lbins_valid = false;
  long long nC = std::max(want, s->lbin_cap);
  free_light_bins(s);
  long long nb = (P + 4095) / 4096;
  if (dalloc(&s->d_lviews, (size_t)s->nl) != cudaSuccess || dalloc(&s->lbin_start, (size_t)P + 1) != cudaSuccess ||
      dalloc(&s->lbin_cur, (size_t)P) != cudaSuccess || dalloc(&s->lbin_list, (size_t)nC) != cudaSuccess ||
      dalloc(&s->lbin_ok, (size_t)s->nl) != cudaSuccess || dalloc(&s->lbin_part, (size_t)nb) != cudaSuccess) {
    free_light_bins(s);
    cudaGetLastError();
    return fail(ST_ERR_OOM, "point-light shadow lists");
  }
  if (!s->lbin_total_host) cudaMallocHost((void**)&s->lbin_total_host, sizeof(int));
  if (s->lbin_total_host) *s->lbin_total_host = 0;
  s->lbin_cells = P;
  s->lbin_cap = nC;
  return ST_OK;
}

// what the bins depend on besides the vertices: each view's camera frame, size and cell layout (bit patterns)
std::vector<uint32_t> bins_key(const Plan& p) {
  std::vector<uint32_t> k;
  auto f = [&](float x) { uint32_t u; std::memcpy(&u, &x, 4); k.push_back(u); };
  for (const DevView& v : p.views) {
    for (const float3& a : {v.eye, v.fwd, v.right, v.up}) { f(a.x); f(a.y); f(a.z); }
    f(v.kx); f(v.ky);
    k.push_back((uint32_t)v.W); k.push_back((uint32_t)v.H); k.push_back((uint32_t)v.kb);
    k.push_back((uint32_t)v.bin_cell); k.push_back((uint32_t)(v.bin_cell >> 32));
  }
  return k;
}

KCtx make_ctx(st_scene* s, const Plan& p) {
  KCtx c;
  c.V = s->verts; c.F = s->faces; c.P = s->params; c.nodes = s->nodes4; c.tri = s->tri; c.nf = s->nf; c.n4 = s->n4;
  c.lights = s->lights; c.nl = s->nl; c.nlt = s->nl + p.max_vl; c.NS = c.nlt + (s->env.w > 0 ? 1 : 0);
  c.env = s->env; c.brdf = s->brdf; c.fresnel = s->fresnel; c.res = s->res; c.ntex = s->ntex; c.np = s->np;
  c.edge_v = s->edge_v; c.edge_f = s->edge_f; c.n_edges = s->n_edges; c.edge_mode = p.o.edge_mode;
  c.edge_flag = s->edge_flag; c.edge_cand = s->edge_cand; c.edge_ncand = s->edge_ncand;
  c.sh_cand = s->sh_cand; c.sh_ncand = s->sh_ncand;
  c.bin_start = p.bins ? s->bin_start : nullptr;   // nullptr: every primary ray traverses the BVH
  c.lviews = s->d_lviews;
  c.lbin_start = p.lbins ? s->lbin_start : nullptr;   // nullptr: every shadow ray traverses the BVH
  c.lbin_list = s->lbin_list; c.lbin_ok = s->lbin_ok; c.lbin_cap = s->lbin_cap; c.lbin_cells = s->lbin_cells;
  c.bin_list = s->bin_list; c.bin_cur = s->bin_cur; c.bin_ok = s->bin_ok;
  c.bin_cap = s->bin_cap; c.bin_pixels = p.pixels; c.bin_cells = p.cells;
  c.cull = s->closed ? 1 : 0; c.mstat = s->mstat;
  c.smooth = s->smooth ? 1 : 0; c.vn = s->vnrm; c.dN = s->dN; c.nv = s->nv;
  c.sec_tree = p.sec_tree ? 1 : 0; c.et_G = s->et_G; c.et_L = s->et_L; c.et_lo = s->et_lo; c.et_hi = s->et_hi;
  c.et_cn = s->et_cn;
  c.acc = s->acc;
  c.views = s->d_views; c.segs = s->d_segs; c.n_segs = (int)p.segs.size();
  c.args = s->d_args; c.B = p.B; c.e = s->eng; c.e.records = p.kind == 1; c.err = s->d_err;
  c.sec = p.sec ? 1 : 0;
  c.sig = p.sig ? 1 : 0; c.sacc = s->sacc;
  return c;
}

int grid_of(const void* fn, int block, int sm) {
  int per = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, block, 0);
  return std::max(1, per) * std::max(1, sm);
}

// event of timed set k (see st_scene::ev): the start of a new pair, or the end of the open one
cudaEvent_t next_event(st_scene* s, int k, bool start) {
  auto& ev = s->ev[k];
  int& used = s->ev_used[k];
  if (used >= (int)ev.size()) {
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    ev.push_back({a, b});
  }
  auto& pr = ev[used];
  if (!start) used++;
  return start ? pr.first : pr.second;
}

// Does any segment of kind k overlap [a, b)?
bool overlaps(const Plan& p, int kind, long long a, long long b) {
  for (auto& sg : p.segs)
    if (sg.kind == kind && sg.base < b && sg.base + sg.count > a) return true;
  return false;
}

// Enqueue one chunk [j0, j0 + n) of the job space. host_sized: read the queue
// counts after each stage and size each grid to them (plain per-view path).
st_status run_chunk(st_scene* s, const Plan& p, const KCtx& c, long long j0, int n, cudaStream_t st, bool host_sized,
                    bool timing, bool has_cam, bool has_edge, cudaEvent_t resolve_after = nullptr,
                    cudaEvent_t resolved = nullptr) {
  int sm = s->sm_count;
  // occupancy-limited grids of the persistent stage kernels, for the scene's own device (a scene is used by one
  // thread at a time, so these per-scene fields need no lock)
  if (!s->g_ext) {
    s->g_ext = grid_of((const void*)k_extend<false>, EXT_BLOCK, sm);
    s->g_ext_s = grid_of((const void*)k_extend<true>, EXT_BLOCK, sm);
    s->g_shade = grid_of((const void*)k_shade, 256, sm);
    s->g_shadow = grid_of((const void*)k_shadow<false>, EXT_BLOCK, sm);
    s->g_shadow_s = grid_of((const void*)k_shadow<true>, EXT_BLOCK, sm);
  }
  const int g_ext = s->g_ext, g_ext_s = s->g_ext_s, g_shade = s->g_shade;
  const int g_shadow = p.o.count_visits ? s->g_shadow_s : s->g_shadow;
  // persistent grids: occupancy limit, or fewer resident blocks per SM if asked
  auto cap = [&](int g) { return p.o.persist_blocks > 0 ? std::min(g, p.o.persist_blocks * sm) : g; };
  int* cnt = c.e.cnt;
  int hc[CNT_SIZE];
  // per-view calls read the queue counts back: the GPU idles from each read until the next launch. With timing on,
  // event pairs bracket the GPU-side intervals between those reads (set 2).
  auto read_counts = [&]() -> st_status {
    if (timing) ST_CUDA(cudaEventRecord(next_event(s, 2, false), st));
    ST_CUDA(copy_async(hc, cnt, sizeof(hc), cudaMemcpyDeviceToHost, st));
    ST_CUDA(cudaStreamSynchronize(st));
    s->host_syncs++;
    if (timing) ST_CUDA(cudaEventRecord(next_event(s, 2, true), st));
    return ST_OK;
  };
  auto shadow = [&](const KCtx& k, int b, int g) -> st_status {
    if (timing) ST_CUDA(cudaEventRecord(next_event(s, 1, true), st));
    if (p.o.count_visits) k_shadow<true><<<g, EXT_BLOCK, 0, st>>>(k, b);
    else k_shadow<false><<<g, EXT_BLOCK, 0, st>>>(k, b);
    if (timing) ST_CUDA(cudaEventRecord(next_event(s, 1, false), st));
    s->launches++;
    return ST_OK;
  };
  // extension / shading / shadow stages for `nb` bounces of the paths queued in q0. With `from_raygen` the first
  // rays already hold their closest hits where a bin cell served them (k_raygen), and bounce 0's BVH launch takes
  // the rest from the fallback queue.
  auto bounces = [&](const KCtx& k, int nb, bool from_raygen) -> st_status {
    for (int b = 0; b < nb; ++b) {
      int ge = cap(p.o.count_visits ? g_ext_s : g_ext), gs = cap(g_shade), gw = cap(g_shadow);
      const bool fb = b == 0 && from_raygen;
      bool launch = true;
      if (host_sized) {
        st_status r = read_counts();
        if (r != ST_OK) return r;
        int q = hc[CNT_EXT + b];
        if (q == 0) break;
        int qe = fb ? hc[CNT_FB] : q;
        launch = qe > 0;
        ge = std::max(1, (qe + EXT_BLOCK - 1) / EXT_BLOCK);
        gs = (q + 255) / 256;
      }
      Range rb(b == 0 ? "bounce 0" : b == 1 ? "bounce 1" : "bounce 2+");
      if (launch) {
        if (timing) ST_CUDA(cudaEventRecord(next_event(s, 0, true), st));
        if (p.o.count_visits) k_extend<true><<<ge, EXT_BLOCK, 0, st>>>(k, b, fb ? 1 : 0);
        else k_extend<false><<<ge, EXT_BLOCK, 0, st>>>(k, b, fb ? 1 : 0);
        if (timing) ST_CUDA(cudaEventRecord(next_event(s, 0, false), st));
        s->launches++;
      }
      k_shade<<<gs, 256, 0, st>>>(k, b);
      s->launches++;
      if (host_sized) {
        st_status r = read_counts();
        if (r != ST_OK) return r;
        int q = hc[CNT_SH + b];
        gw = (q + EXT_BLOCK - 1) / EXT_BLOCK;
        if (q > 0) {
          r = shadow(k, b, gw);
          if (r != ST_OK) return r;
        }
      } else if (k.NS > 0) {
        st_status r = shadow(k, b, gw);
        if (r != ST_OK) return r;
      }
    }
    return ST_OK;
  };
  Range rc("chunk");
  k_reset<<<1, 128, 0, st>>>(cnt);
  bool has_shadow = p.shadow && overlaps(p, 2, j0, j0 + n);
  if (has_shadow) { k_sh_prep<<<(n + EXT_BLOCK - 1) / EXT_BLOCK, EXT_BLOCK, 0, st>>>(c, j0, n); s->launches++; }
  // k_raygen finds the closest hits of the first rays its bin cells serve: timed with the closest-hit launches
  {
    const int gr = (n + 255) / 256;
    if (timing) ST_CUDA(cudaEventRecord(next_event(s, 0, true), st));
    if (has_shadow) {
      if (p.o.count_visits) k_raygen<true, true><<<gr, 256, 0, st>>>(c, j0, n);
      else k_raygen<true, false><<<gr, 256, 0, st>>>(c, j0, n);
    } else {
      if (p.o.count_visits) k_raygen<false, true><<<gr, 256, 0, st>>>(c, j0, n);
      else k_raygen<false, false><<<gr, 256, 0, st>>>(c, j0, n);
    }
    if (timing) ST_CUDA(cudaEventRecord(next_event(s, 0, false), st));
    s->launches += 2;
  }
  st_status r = bounces(c, p.B, true);
  if (r != ST_OK) return r;
  Range rr(p.kind == 0 ? "resolve" : "adjoint");
  if (p.kind == 0) {
    // pixels add their samples in sample order: this chunk's sums come after the previous chunk's
    if (resolve_after) ST_CUDA(cudaStreamWaitEvent(st, resolve_after, 0));
    k_resolve<<<(n + RESOLVE_BLOCK - 1) / RESOLVE_BLOCK, RESOLVE_BLOCK, 0, st>>>(c, j0, n);
    if (resolved) ST_CUDA(cudaEventRecord(resolved, st));
    s->launches++;
  } else {
    int ga = (n + ADJ_BLOCK - 1) / ADJ_BLOCK;
    if (has_edge) { k_edge_resolve<<<ga, ADJ_BLOCK, 0, st>>>(c, j0, n); s->launches++; }
    if (has_shadow) { k_sh_resolve<<<(n + 255) / 256, 256, 0, st>>>(c, j0, n); s->launches++; }
    if (has_cam && p.sec) {
      // secondary edge samples: jobs from the recorded vertices, then their side
      // paths in passes of Q slots (records off: they stay the camera paths'),
      // each pass resolved before the next reuses the slots
      k_sec_gen<<<ga, ADJ_BLOCK, 0, st>>>(c, j0, n);
      s->launches++;
      long long jobs = (long long)p.B * n;
      if (host_sized) {
        r = read_counts();
        if (r != ST_OK) return r;
        jobs = hc[CNT_SEC];
      }
      int Q = c.e.Q;
      long long sides = (jobs + 31) / 32 * 64;
      int passes = (int)((sides + Q - 1) / Q);
      KCtx cs = c;
      cs.e.records = false;
      for (int ps = 0; ps < passes; ++ps) {
        k_reset_pass<<<1, 128, 0, st>>>(cnt);
        Range rs("secondary edge pass");
        k_sec_raygen<<<std::min((Q + 255) / 256, 4 * sm), 256, 0, st>>>(cs, ps);
        s->launches += 2;
        r = bounces(cs, std::max(1, p.B - 1), false);
        if (r != ST_OK) return r;
        k_sec_resolve<<<std::min((Q + ADJ_BLOCK - 1) / ADJ_BLOCK, 8 * sm), ADJ_BLOCK, 0, st>>>(cs, ps);
        s->launches++;
      }
    }
    if (has_cam && p.interior) {
      if (s->smooth) k_adjoint<true><<<ga, ADJ_BLOCK, 0, st>>>(c, j0, n);
      else k_adjoint<false><<<ga, ADJ_BLOCK, 0, st>>>(c, j0, n);
      s->launches++;
    }
  }
  ST_CUDA(cudaGetLastError());
  return ST_OK;
}


st_status enqueue_body(st_scene* s, const Plan& p, const KCtx& c, int Q, cudaStream_t st, bool host_sized,
                       bool timing);

long long chunk_count(const Plan& p, int Q) {
  if (p.o.mode == ST_MODE_PER_VIEW) return 0;
  return (p.total + Q - 1) / Q;
}

// Overlap consecutive chunks on the engines: batched calls of two chunks or more whose grids are not sized on the
// host and whose kernels are not timed one by one, once the further engines and the events are in place.
bool overlap_chunks(const st_scene* s, const Plan& p, int Q, bool host_sized, bool timing) {
  long long nc = chunk_count(p, Q);
  if (host_sized || timing || nc < 2 || (long long)s->xev.size() < nc + 2 * OVERLAP_ENGINES) return false;
  for (int k = 0; k < OVERLAP_ENGINES - 1; ++k)
    if (!s->aux_stream[k] || s->eng2[k].Q < Q || s->eng2[k].records != s->eng.records) return false;
  return true;
}

st_status enqueue_call(st_scene* s, const Plan& p, int Q, cudaStream_t st, bool host_sized, bool timing) {
  KCtx c = make_ctx(s, p);
  if (timing) ST_CUDA(cudaEventRecord(next_event(s, 2, true), st));
  st_status body = enqueue_body(s, p, c, Q, st, host_sized, timing);
  if (timing) ST_CUDA(cudaEventRecord(next_event(s, 2, false), st));
  return body;
}

st_status enqueue_body(st_scene* s, const Plan& p, const KCtx& c, int Q, cudaStream_t st, bool host_sized,
                       bool timing) {
  ST_CUDA(cudaMemsetAsync(s->eng.stat, 0, sizeof(unsigned long long) * STAT_SIZE, st));
  for (auto& e : s->eng2)
    if (e.stat) ST_CUDA(cudaMemsetAsync(e.stat, 0, sizeof(unsigned long long) * STAT_SIZE, st));
  if (p.kind == 0) {
    k_zero_acc<<<(unsigned)((p.pixels + 255) / 256), 256, 0, st>>>(c);
    s->launches++;
  }
  if (p.kind == 1 && s->smooth) ST_CUDA(cudaMemsetAsync(s->dN, 0, 3 * sizeof(float) * s->nv, st));
  if (p.sec_tree) {
    // the edge hierarchy on the current vertices: leaves, then level by level up to the root
    int nl = 1 << s->et_L;
    k_etree_leaves<<<std::min((nl + 255) / 256, 4 * std::max(s->sm_count, 1)), 256, 0, st>>>(c, s->et_lo, s->et_hi,
                                                                                             s->et_cn);
    for (int l = s->et_L - 1; l >= 0; --l)
      k_etree_level<<<std::min(((1 << l) + 255) / 256, 4 * std::max(s->sm_count, 1)), 256, 0, st>>>(
          s->et_lo, s->et_hi, s->et_cn, l);
    s->launches += 1 + s->et_L;
  }
  if (p.bins && !p.bins_reused) {
    Range r("primary bins");
    // primary-visibility bins of every view: count, scan, fill
    long long P = p.cells;
    int nv = (int)p.views.size();
    long long nb = (P + 4095) / 4096;
    dim3 g((s->nf + 127) / 128, (unsigned)nv);
    ST_CUDA(cudaMemsetAsync(s->bin_cur, 0, sizeof(int) * P, st));
    k_fill_int<<<(nv + 127) / 128, 128, 0, st>>>(s->bin_ok, nv, 1);
    k_bin<0><<<g, 128, 0, st>>>(c, nv, s->bin_ok);
    k_scan_blocks<<<(unsigned)nb, SCAN_BLOCK, 0, st>>>(s->bin_cur, s->bin_start, P, s->bin_part);
    k_scan_parts<<<1, SCAN_BLOCK, 0, st>>>(s->bin_part, (int)nb, s->bin_start, P);
    k_scan_add<<<(unsigned)nb, SCAN_BLOCK, 0, st>>>(s->bin_start, P, s->bin_part);
    ST_CUDA(cudaMemsetAsync(s->bin_cur, 0, sizeof(int) * P, st));
    k_bin<1><<<g, 128, 0, st>>>(c, nv, s->bin_ok);
    ST_CUDA(copy_async(s->bin_total_host, s->bin_start + P, sizeof(int), cudaMemcpyDeviceToHost, st));
    s->launches += 6;
  }
  if (p.lbins && !p.lbins_reused) {
    Range r("light bins");
    // a frustum per scene light from the current vertex bounds, then count, scan and fill as for the views
    const int nl = s->nl;
    const long long P = s->lbin_cells;
    const long long nb = (P + 4095) / 4096;
    KCtx cl = c;
    cl.views = s->d_lviews;
    cl.bin_start = s->lbin_start; cl.bin_list = s->lbin_list; cl.bin_cur = s->lbin_cur; cl.bin_ok = s->lbin_ok;
    cl.bin_cap = s->lbin_cap; cl.bin_cells = P;
    dim3 g((s->nf + 127) / 128, (unsigned)nl);
    k_fill_int<<<(nl + 127) / 128, 128, 0, st>>>(s->lbin_ok, nl, 1);
    k_light_views<<<nl, LVIEW_BLOCK, 0, st>>>(s->lights, s->verts, s->nv, s->mstat, s->lbin_res, s->d_lviews,
                                             s->lbin_ok);
    ST_CUDA(cudaMemsetAsync(s->lbin_cur, 0, sizeof(int) * P, st));
    k_bin<0><<<g, 128, 0, st>>>(cl, nl, s->lbin_ok);
    k_scan_blocks<<<(unsigned)nb, SCAN_BLOCK, 0, st>>>(s->lbin_cur, s->lbin_start, P, s->lbin_part);
    k_scan_parts<<<1, SCAN_BLOCK, 0, st>>>(s->lbin_part, (int)nb, s->lbin_start, P);
    k_scan_add<<<(unsigned)nb, SCAN_BLOCK, 0, st>>>(s->lbin_start, P, s->lbin_part);
    ST_CUDA(cudaMemsetAsync(s->lbin_cur, 0, sizeof(int) * P, st));
    k_bin<1><<<g, 128, 0, st>>>(cl, nl, s->lbin_ok);
    ST_CUDA(copy_async(s->lbin_total_host, s->lbin_start + P, sizeof(int), cudaMemcpyDeviceToHost, st));
    s->launches += 7;
  }
  if (p.shadow && !p.pairs.empty()) {
    int np = (int)p.pairs.size();
    dim3 g((s->n_edges + 255) / 256, (unsigned)np);
    k_sh_flags<<<g, 256, 0, st>>>(c, s->d_pairs, np, s->sh_flag);
    KCtx cc = c;   // the ordered compaction of the primary candidates, on the shadow tables
    cc.edge_flag = s->sh_flag; cc.edge_cand = s->sh_cand; cc.edge_ncand = s->sh_ncand;
    k_edge_compact<<<(unsigned)np, 1024, 0, st>>>(cc);
    s->launches += 2;
  }
  if (p.edges) {
    Range r("edge candidates");
    dim3 g((s->n_edges + 255) / 256, (unsigned)p.views.size());
    k_edge_flags<<<g, 256, 0, st>>>(c, (int)p.views.size());
    k_edge_compact<<<(unsigned)p.views.size(), 1024, 0, st>>>(c);
    s->launches += 2;
  }
  // Batched calls of several chunks rotate them over the engines, each on its own
  // stream, so one chunk's last, sparsely filled bounces and launch tails overlap
  // the next chunks' full stages. The auxiliary streams fork after the set-up
  // above and join before the finishing kernels; forward chunks resolve in order.
  const bool multi = overlap_chunks(s, p, Q, host_sized, timing);
  KCtx cx[OVERLAP_ENGINES];
  cudaStream_t sx[OVERLAP_ENGINES];
  cx[0] = c;
  sx[0] = st;
  for (int k = 1; k < OVERLAP_ENGINES; ++k) {
    cx[k] = c;
    cx[k].e = s->eng2[k - 1];
    cx[k].e.records = c.e.records;
    sx[k] = s->aux_stream[k - 1];
  }
  auto chunks = [&](long long a, long long b) -> st_status {
    cudaEvent_t prev = nullptr;
    int k = 0;
    if (multi) {
      cudaEvent_t fork = s->xev[s->xev_used++];
      ST_CUDA(cudaEventRecord(fork, st));
      for (int i = 1; i < OVERLAP_ENGINES; ++i) ST_CUDA(cudaStreamWaitEvent(sx[i], fork, 0));
    }
    for (long long j0 = a; j0 < b; j0 += Q, ++k) {
      int n = (int)std::min<long long>(Q, b - j0);
      int e = multi ? k % OVERLAP_ENGINES : 0;
      cudaEvent_t done = multi && p.kind == 0 ? s->xev[s->xev_used++] : nullptr;
      st_status r = run_chunk(s, p, cx[e], j0, n, sx[e], host_sized, timing, overlaps(p, 0, j0, j0 + n),
                              overlaps(p, 1, j0, j0 + n), prev, done);
      if (r != ST_OK) return r;
      prev = done;
    }
    if (multi) {
      for (int i = 1; i < OVERLAP_ENGINES; ++i) {
        cudaEvent_t join = s->xev[s->xev_used++];
        ST_CUDA(cudaEventRecord(join, sx[i]));
        ST_CUDA(cudaStreamWaitEvent(st, join, 0));
      }
    }
    return ST_OK;
  };
  if (p.o.mode == ST_MODE_PER_VIEW) {
    for (auto& r : p.view_range) {
      st_status x = chunks(r.first, r.second);
      if (x != ST_OK) return x;
    }
  } else {
    st_status x = chunks(0, p.total);
    if (x != ST_OK) return x;
  }
  if (p.kind == 0) {
    k_finish_views<<<(unsigned)((p.pixels + 255) / 256), 256, 0, st>>>(c, (int)p.views.size());
    s->launches++;
    ST_CUDA(cudaGetLastError());
  }
  if (p.kind == 1 && s->smooth) {
    int g = std::min((std::max(s->nv, s->nf) + 255) / 256, 4 * std::max(s->sm_count, 1));
    k_vn_adj_vertex<<<g, 256, 0, st>>>(c);
    k_vn_adj_face<<<g, 256, 0, st>>>(c);
    s->launches += 2;
    ST_CUDA(cudaGetLastError());
  }
  return ST_OK;
}

std::vector<long long> graph_key(const Plan& p, int Q, const st_scene* s) {
  std::vector<long long> k = {p.kind, p.B, (long long)p.views.size(), Q, p.o.edge_term, p.o.edge_mode, p.o.edge_spp,
                              p.interior, p.edges, p.o.count_visits, p.bins, p.bins_reused, p.lbins,
                              p.lbins_reused, s->lbin_cap,
                              p.o.persist_blocks, s->bin_cap, p.max_vl, p.sig, p.sec_tree};
  for (auto& v : p.views) {
    k.push_back(v.W); k.push_back(v.H); k.push_back(v.spp); k.push_back(v.pix_off); k.push_back(v.nvl);
  }
  return k;
}

st_status plan_call(st_scene* s, const st_view* views, int n_views, int default_spp, int B, const st_render_opts* opts,
                    int kind, bool want_interior, Plan& p) {
  if (!views || n_views <= 0) return fail(ST_ERR_INVALID_ARG, "no views");
  if (n_views > ST_MAX_VIEWS) return fail(ST_ERR_UNSUPPORTED, "more than ST_MAX_VIEWS views in one call");
  if (B < 1 || B > ST_MAX_BOUNCES) return fail(ST_ERR_UNSUPPORTED, "max_bounces must be in [1, 8]");
  p.kind = kind;
  p.B = B;
  p.o = opts ? *opts : default_opts();
  if (p.o.mode != ST_MODE_BATCHED && p.o.mode != ST_MODE_PER_VIEW) return fail(ST_ERR_INVALID_ARG, "bad mode");
  if (p.o.edge_mode != ST_EDGE_SILHOUETTE && p.o.edge_mode != ST_EDGE_ALL) return fail(ST_ERR_INVALID_ARG, "bad edge_mode");
  if (p.o.edge_spp < 0 || p.o.chunk_paths < 0 || p.o.persist_blocks < 0)
    return fail(ST_ERR_INVALID_ARG, "negative option");
  if (p.o.edge_term < 0 || p.o.edge_term > (ST_EDGE_TERM_PRIMARY | ST_EDGE_TERM_SECONDARY | ST_EDGE_TERM_SHADOW))
    return fail(ST_ERR_INVALID_ARG, "bad edge_term");
  p.sig = kind == 0 && p.o.path_signatures != nullptr;
  p.interior = kind == 1 && want_interior;
  p.edges = kind == 1 && (p.o.edge_term & ST_EDGE_TERM_PRIMARY);
  p.sec = p.interior && (p.o.edge_term & ST_EDGE_TERM_SECONDARY) && s->n_edges > 0;
  if (p.o.sec_pick != ST_SEC_PICK_TREE && p.o.sec_pick != ST_SEC_PICK_UNIFORM) return fail(ST_ERR_INVALID_ARG, "bad sec_pick");
  p.sec_tree = p.sec && p.o.sec_pick == ST_SEC_PICK_TREE;
  p.shadow = kind == 1 && (p.o.edge_term & ST_EDGE_TERM_SHADOW) && s->n_edges > 0;
  long long base = 0;
  for (int i = 0; i < n_views; ++i) {
    const st_view& v = views[i];
    if (!view_ok(v)) return fail(ST_ERR_INVALID_ARG, "view " + std::to_string(i) + " is invalid");
    if (v.n_lights < 0 || v.n_lights > ST_MAX_VIEW_LIGHTS || s->nl + v.n_lights > ST_MAX_LIGHTS)
      return fail(ST_ERR_INVALID_ARG, "view " + std::to_string(i) + ": bad number of view lights");
    for (int j = 0; j < v.n_lights; ++j)
      for (int k = 0; k < 3; ++k)
        if (!std::isfinite(v.lights[j].pos[k]) || !std::isfinite(v.lights[j].intensity[k]) ||
            v.lights[j].intensity[k] < 0.0f)
          return fail(ST_ERR_INVALID_ARG, "view " + std::to_string(i) + ": bad view light");
    p.max_vl = std::max(p.max_vl, v.n_lights);
    int spp = v.spp > 0 ? v.spp : default_spp;
    if (spp <= 0) return fail(ST_ERR_INVALID_ARG, "view " + std::to_string(i) + " has no samples");
    if ((long long)v.width * v.height > (1LL << 31) || v.pixel_offset + (long long)v.width * v.height > (1LL << 32))
      return fail(ST_ERR_UNSUPPORTED, "view too large for 32-bit pixel counters");
    p.views.push_back(make_view(v, spp));
    p.views.back().bin_base = p.pixels;
    p.pixels += (long long)v.width * v.height;
    {
      // bin cells per pixel side: enough that a cell holds a few faces when the mesh is dense on screen (a
      // 64 x 64 view of 200,000 faces gets 8 x 8 cells per pixel), at most 8
      int kb = 1;
      while (kb < 8 && (double)s->nf > BIN_FACES_PER_CELL * (double)v.width * v.height * kb * kb) kb *= 2;
      p.views.back().kb = kb;
      p.views.back().bin_cell = p.cells;
      p.cells += (long long)v.width * v.height * kb * kb;
    }
    long long start = base;
    long long cam = (long long)v.width * v.height * spp;
    if (kind == 0 || p.interior) {
      Seg sg{base, cam, i, 0, 0, 0, cam};
      p.segs.push_back(sg);
      base += (cam + SEG_ALIGN - 1) / SEG_ALIGN * SEG_ALIGN;
    }
    if (p.edges) {
      long long ne = (long long)v.width * v.height * (p.o.edge_spp > 0 ? p.o.edge_spp : spp);
      Seg sg{base, (ne + 31) / 32 * 64, i, 1, 0, 0, ne};
      p.segs.push_back(sg);
      base += sg.count;
    }
    if (p.shadow) {
      long long ne = (long long)v.width * v.height * (p.o.edge_spp > 0 ? p.o.edge_spp : spp);
      for (int l = 0; l < s->nl + v.n_lights; ++l) {
        if (p.pairs.size() >= (size_t)ST_MAX_VIEWS)
          return fail(ST_ERR_UNSUPPORTED, "shadow edges: more than ST_MAX_VIEWS (view, light) pairs in one call");
        Seg sg{base, (ne + 31) / 32 * 64, i, 2, (unsigned)l, (unsigned)p.pairs.size(), ne};
        p.pairs.push_back(make_int2(i, l));
        p.segs.push_back(sg);
        base += sg.count;
      }
    }
    p.view_range.push_back({start, base});
  }
  p.total = base;
  if (s->nl == 0 && s->env.w == 0 && p.max_vl == 0)
    return fail(ST_ERR_INVALID_ARG, "no light: the scene has none and no view brings one");
  // below about a million primary rays the fixed cost of building the bins
  // (seven launches) exceeds what they save; those calls traverse the BVH
  p.bins = p.total >= (1LL << 20);
  p.lbins = p.bins && s->nl > 0;   // the same threshold: the build is a few launches over the faces
  {
    std::vector<std::pair<long long, long long>> rg;
    for (int i = 0; i < n_views; ++i)
      rg.push_back({views[i].pixel_offset, views[i].pixel_offset + (long long)views[i].width * views[i].height});
    std::sort(rg.begin(), rg.end());
    for (size_t i = 1; i < rg.size(); ++i)
      if (rg[i].first < rg[i - 1].second) return fail(ST_ERR_INVALID_ARG, "views' pixel ranges overlap");
  }
  s->last_edge_samples = 0;
  for (auto& sg : p.segs)
    if (sg.kind == 1) s->last_edge_samples += sg.n_samples;
  return ST_OK;
}

st_status launch_call(st_scene* s, Plan& p, const CallArgs& args, int Q, cudaStream_t st);

st_status run_call(st_scene* s, Plan& p, const CallArgs& args, cudaStream_t st) {
  st_status r = ensure_tables(s, (int)p.views.size(), (int)p.segs.size(), p.edges);
  if (r != ST_OK) return r;
  if (p.shadow && (int)p.pairs.size() > s->sh_cap_pairs) {
    cudaDeviceSynchronize();
    drop_graphs(s);
    dfree(s->sh_flag); dfree(s->sh_cand); dfree(s->sh_ncand); dfree(s->d_pairs);
    size_t n = p.pairs.size() * (size_t)std::max(s->n_edges, 1);
    if (dalloc(&s->sh_flag, n) != cudaSuccess || dalloc(&s->sh_cand, n) != cudaSuccess ||
        dalloc(&s->sh_ncand, p.pairs.size()) != cudaSuccess || dalloc(&s->d_pairs, p.pairs.size()) != cudaSuccess) {
      dfree(s->sh_flag); dfree(s->sh_cand); dfree(s->sh_ncand); dfree(s->d_pairs);
      cudaGetLastError();
      s->sh_cap_pairs = 0;
      return fail(ST_ERR_OOM, "shadow-edge tables");
    }
    s->sh_cap_pairs = (int)p.pairs.size();
  }
  std::vector<uint32_t> bkey;
  if (p.bins) {
    r = ensure_bins(s, p);
    if (r != ST_OK) return r;
    bkey = bins_key(p);
    // a build whose lists overflowed (as far as its readback shows yet) is redone with more room
    p.bins_reused = s->bins_valid && s->bins_geom == s->geom_version && s->bins_key == bkey &&
                    !(s->bin_total_host && *s->bin_total_host > s->bin_cap);
    if (!p.bins_reused) s->bins_valid = false;
  }
  if (p.lbins) {
    r = ensure_light_bins(s);
    if (r != ST_OK) return r;
    p.lbins_reused = s->lbins_valid && s->lbins_geom == s->geom_version &&
                     !(s->lbin_total_host && *s->lbin_total_host > s->lbin_cap);
    if (!p.lbins_reused) s->lbins_valid = false;
  }
  if (p.kind == 0 && p.pixels > s->acc_cap) {
    cudaDeviceSynchronize();
    drop_graphs(s);
    dfree(s->acc);
    dfree(s->sacc);
    if (dalloc(&s->acc, 6 * (size_t)p.pixels) != cudaSuccess || dalloc(&s->sacc, (size_t)p.pixels) != cudaSuccess) {
      dfree(s->acc);
      dfree(s->sacc);
      cudaGetLastError();
      s->acc_cap = 0;
      return fail(ST_ERR_OOM, "forward accumulation buffer");
    }
    s->acc_cap = p.pixels;
  }
  long long Q64 = p.o.chunk_paths > 0 ? p.o.chunk_paths : DEFAULT_CHUNK;
  Q64 = std::min<long long>(Q64, std::max<long long>(p.total, SEG_ALIGN));
  Q64 = (Q64 + SEG_ALIGN - 1) / SEG_ALIGN * SEG_ALIGN;
  int Q = (int)Q64;
  if (p.o.mode == ST_MODE_PER_VIEW) {
    long long mx = SEG_ALIGN;
    for (auto& vr : p.view_range) mx = std::max(mx, vr.second - vr.first);
    Q = (int)std::min<long long>(Q, (mx + SEG_ALIGN - 1) / SEG_ALIGN * SEG_ALIGN);
  }
  int NS = s->nl + p.max_vl + (s->env.w > 0 ? 1 : 0);
  bool timing_call = p.o.time_kernels != 0;
  bool want_two = p.o.mode == ST_MODE_BATCHED && !timing_call && chunk_count(p, Q) >= 2;
  r = ensure_engine(s, Q, p.B, NS, p.kind == 1, p.sec, p.shadow, want_two);
  if (r != ST_OK) return r;
  if (want_two) {
    // events for the fork, every chunk's resolve and the join, made before any capture
    long long need = chunk_count(p, Q) + 2 * OVERLAP_ENGINES;
    while ((long long)s->xev.size() < need) {
      cudaEvent_t e;
      ST_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
      s->xev.push_back(e);
    }
  }
  st_status res = launch_call(s, p, args, Q, st);
  if (res == ST_OK && p.bins && !p.bins_reused) {
    s->bins_valid = true;
    s->bins_geom = s->geom_version;
    s->bins_key = std::move(bkey);
  }
  if (res == ST_OK && p.lbins && !p.lbins_reused) {
    s->lbins_valid = true;
    s->lbins_geom = s->geom_version;
  }
  return res;
}

// upload the call's tables and enqueue it: directly, or as the replay of a graph captured once per call shape
st_status launch_call(st_scene* s, Plan& p, const CallArgs& args, int Q, cudaStream_t st) {
  s->xev_used = 0;
  ST_CUDA(copy_async(s->d_views, p.views.data(), sizeof(DevView) * p.views.size(), cudaMemcpyHostToDevice, st));
  ST_CUDA(copy_async(s->d_segs, p.segs.data(), sizeof(Seg) * p.segs.size(), cudaMemcpyHostToDevice, st));
  if (p.shadow && !p.pairs.empty())
    ST_CUDA(copy_async(s->d_pairs, p.pairs.data(), sizeof(int2) * p.pairs.size(), cudaMemcpyHostToDevice, st));
  ST_CUDA(copy_async(s->d_args, &args, sizeof(CallArgs), cudaMemcpyHostToDevice, st));
  bool timing = p.o.time_kernels != 0;
  for (int k = 0; k < 3; ++k) s->ev_used[k] = 0;
  s->host_syncs = 0;
  s->launches = 0;
  bool graph = p.o.mode == ST_MODE_BATCHED && p.o.use_graph && !timing;
  if (!graph) return enqueue_call(s, p, Q, st, p.o.mode == ST_MODE_PER_VIEW, timing);
  std::vector<long long> key = graph_key(p, Q, s);
  for (auto& g : s->graphs)
    if (g.key == key) {
      s->launches = g.launches;
      ST_CUDA(cudaGraphLaunch(g.exec, st));
      return ST_OK;
    }
  // capture on the scene's own stream, ordered after the uploads above
  cudaEvent_t ready;
  ST_CUDA(cudaEventCreateWithFlags(&ready, cudaEventDisableTiming));
  ST_CUDA(cudaEventRecord(ready, st));
  ST_CUDA(cudaStreamWaitEvent(s->cap_stream, ready, 0));
  ST_CUDA(cudaStreamSynchronize(s->cap_stream));
  cudaEventDestroy(ready);
  ST_CUDA(cudaStreamBeginCapture(s->cap_stream, cudaStreamCaptureModeThreadLocal));
  st_status er = enqueue_call(s, p, Q, s->cap_stream, false, false);
  cudaGraph_t graph_obj = nullptr;
  cudaError_t ce = cudaStreamEndCapture(s->cap_stream, &graph_obj);
  if (er != ST_OK) {
    if (graph_obj) cudaGraphDestroy(graph_obj);
    return er;
  }
  if (ce != cudaSuccess) return cuda_fail(ce, "cudaStreamEndCapture");
  GraphEntry ge;
  ge.key = key;
  ge.launches = s->launches;
  ce = cudaGraphInstantiate(&ge.exec, graph_obj, 0);
  cudaGraphDestroy(graph_obj);
  if (ce != cudaSuccess) return cuda_fail(ce, "cudaGraphInstantiate");
  if (s->graphs.size() >= 16) {
    cudaGraphExecDestroy(s->graphs.front().exec);
    s->graphs.erase(s->graphs.begin());
  }
  s->graphs.push_back(ge);
  ST_CUDA(cudaGraphLaunch(ge.exec, st));
  return ST_OK;
}

void destroy(st_scene* s) {
  if (!s) return;
  cudaSetDevice(s->device);
  cudaDeviceSynchronize();
  drop_graphs(s);
  free_engine(s->eng);
  for (auto& e : s->eng2) free_engine(e);
  dfree(s->verts); dfree(s->faces); dfree(s->params); dfree(s->tri); dfree(s->nodes); dfree(s->parent);
  dfree(s->flags); dfree(s->keys); dfree(s->keys2); dfree(s->ids); dfree(s->ids2); dfree(s->hist); dfree(s->bounds);
  dfree(s->nodes4); dfree(s->src4); dfree(s->q4); dfree(s->c4);
  dfree(s->lights); dfree(s->env_tex); dfree(s->env_alias); dfree(s->edge_v); dfree(s->edge_f);
  dfree(s->edge_flag); dfree(s->edge_cand); dfree(s->edge_ncand);
  dfree(s->sh_flag); dfree(s->sh_cand); dfree(s->sh_ncand); dfree(s->d_pairs); dfree(s->d_views); dfree(s->d_segs);
  free_light_bins(s);
  if (s->lbin_total_host) cudaFreeHost(s->lbin_total_host);
  dfree(s->bin_start); dfree(s->bin_cur); dfree(s->bin_list); dfree(s->bin_ok); dfree(s->bin_part);
  dfree(s->acc); dfree(s->sacc); dfree(s->mstat); dfree(s->vnrm); dfree(s->vf_start); dfree(s->vf_list); dfree(s->dN);
  dfree(s->et_lo); dfree(s->et_hi); dfree(s->et_cn);
  if (s->bin_total_host) cudaFreeHost(s->bin_total_host);
  dfree(s->d_args); dfree(s->d_err);
  for (auto& set : s->ev)
    for (auto& e : set) { cudaEventDestroy(e.first); cudaEventDestroy(e.second); }
  for (auto e : s->xev) cudaEventDestroy(e);
  if (s->cap_stream) cudaStreamDestroy(s->cap_stream);
  for (auto a : s->aux_stream)
    if (a) cudaStreamDestroy(a);
  delete s;
}

// caller texels (np = 5: kd rgb, ks, roughness; np = 7: kd rgb, ks rgb, roughness) to the
// device layout (kd rgb, ks_r), (roughness, ks_g, ks_b, 0)
__global__ void k_params_in(const float* in, float4* out, int nt, int np) {
  int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= nt) return;
  const float* p = in + (size_t)np * f;
  float kg = np == 7 ? p[4] : p[3], kb = np == 7 ? p[5] : p[3];
  out[2 * f] = make_float4(p[0], p[1], p[2], p[3]);
  out[2 * f + 1] = make_float4(p[np - 1], kg, kb, 0.0f);
}

}  // namespace
}  // namespace st

using namespace st;

extern "C" {

const char* st_last_error(void) { return g_err.c_str(); }

st_status st_inject_fault(int site, int nth) {
  if (site != ST_FAULT_ALLOC && site != ST_FAULT_COPY) return fail(ST_ERR_INVALID_ARG, "unknown fault site");
  fault_init();
  g_fault[site].store(nth < 0 ? -1 : nth);
  return ST_OK;
}

st_status st_scene_create(const st_scene_desc* d, void* stream, st_scene** out) {
  if (!out) return fail(ST_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (!d || d->n_vertices <= 0 || d->n_faces <= 0 || !d->vertices || !d->faces || !d->face_params)
    return fail(ST_ERR_INVALID_ARG, "mesh description incomplete");
  if (d->n_faces > (1 << 28)) return fail(ST_ERR_UNSUPPORTED, "too many faces");
  if (d->brdf != ST_BRDF_GGX && d->brdf != ST_BRDF_BECKMANN) return fail(ST_ERR_INVALID_ARG, "unknown brdf");
  if (d->bvh_builder != ST_BVH_PLOC && d->bvh_builder != ST_BVH_LBVH) return fail(ST_ERR_INVALID_ARG, "unknown bvh_builder");
  if (d->color_res < 0 || d->color_res > 64) return fail(ST_ERR_UNSUPPORTED, "mesh-colors resolution must be in [0, 64]");
  if (d->smooth_normals != 0 && d->smooth_normals != 1) return fail(ST_ERR_INVALID_ARG, "smooth_normals must be 0 or 1");
  if (d->fresnel != ST_FRESNEL_HELD && d->fresnel != ST_FRESNEL_SCHLICK) return fail(ST_ERR_INVALID_ARG, "unknown fresnel");
  if ((long long)d->n_faces * (d->color_res + 1) * (d->color_res + 2) / 2 > (1LL << 30))
    return fail(ST_ERR_UNSUPPORTED, "too many mesh-colors texels");
  if (d->n_point_lights < 0 || d->n_point_lights > ST_MAX_LIGHTS || (d->n_point_lights > 0 && !d->point_lights))
    return fail(ST_ERR_INVALID_ARG, "bad point lights");
  for (int j = 0; j < d->n_point_lights; ++j)
    for (int k = 0; k < 3; ++k)
      if (!std::isfinite(d->point_lights[j].pos[k]) || !std::isfinite(d->point_lights[j].intensity[k]) ||
          d->point_lights[j].intensity[k] < 0)
        return fail(ST_ERR_INVALID_ARG, "point light " + std::to_string(j) + " is invalid");
  if (d->env && (d->env->width <= 0 || d->env->height <= 0 || !d->env->rgb ||
                 (long long)d->env->width * d->env->height > (1LL << 24)))
    return fail(ST_ERR_INVALID_ARG, "bad environment map");
  cudaStream_t st = (cudaStream_t)stream;
  st_scene* s = new st_scene();
  cudaGetDevice(&s->device);
  cudaDeviceGetAttribute(&s->sm_count, cudaDevAttrMultiProcessorCount, s->device);
  s->nv = d->n_vertices;
  s->nf = d->n_faces;
  s->brdf = d->brdf;
  s->nl = d->n_point_lights;
  s->res = d->color_res;
  s->builder = d->bvh_builder;
  s->np = d->rgb_specular ? 7 : 5;
  s->smooth = d->smooth_normals == 1;
  s->fresnel = d->fresnel;
  s->ntex = (s->res + 1) * (s->res + 2) / 2;
  // host copy of the faces: validation and edge list
  std::vector<int> hf(3 * (size_t)s->nf);
  std::vector<float> hv(3 * (size_t)s->nv);
  cudaError_t e = copy_async(hf.data(), d->faces, hf.size() * sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = copy_async(hv.data(), d->vertices, hv.size() * sizeof(float), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) { destroy(s); return cuda_fail(e, "reading the mesh"); }
  for (int v : hf)
    if (v < 0 || v >= s->nv) { destroy(s); return fail(ST_ERR_INVALID_ARG, "face index out of range"); }
  for (float x : hv)
    if (!std::isfinite(x)) { destroy(s); return fail(ST_ERR_INVALID_ARG, "non-finite vertex"); }
  for (int f = 0; f < s->nf; ++f) {
    int a = hf[3 * f], b = hf[3 * f + 1], c = hf[3 * f + 2];
    if (a == b || b == c || a == c) { destroy(s); return fail(ST_ERR_INVALID_ARG, "degenerate face " + std::to_string(f)); }
  }
  std::vector<int2> ev, ef;
  build_edges(hf, s->nf, ev, ef);
  s->closed = closed_single_surface(hf, s->nf, ef);
  s->n_edges = (int)ev.size();
  std::vector<float4> etex;
  std::vector<float2> etab;
  if (d->env) {
    // the map may be host or device memory; device memory is read back once (the alias table is built on the host)
    const float* rgb = d->env->rgb;
    std::vector<float> hrgb;
    cudaPointerAttributes pa{};
    cudaError_t pe = cudaPointerGetAttributes(&pa, rgb);
    if (pe != cudaSuccess) cudaGetLastError();
    if (pe == cudaSuccess && pa.type == cudaMemoryTypeDevice) {
      hrgb.resize(3 * (size_t)d->env->width * d->env->height);
      e = copy_async(hrgb.data(), rgb, hrgb.size() * sizeof(float), cudaMemcpyDeviceToHost, st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(st);
      if (e != cudaSuccess) { destroy(s); return cuda_fail(e, "reading the environment map"); }
      rgb = hrgb.data();
    }
    if (!build_alias(rgb, d->env->width, d->env->height, etex, etab)) {
      destroy(s);
      return fail(ST_ERR_INVALID_ARG, "environment map has no positive finite weight");
    }
  }
  int n = s->nf;
  s->sort_blocks = sort_blocks_for(n);
  e = cudaSuccess;
  auto chk = [&](cudaError_t x) { if (x != cudaSuccess && e == cudaSuccess) e = x; };
  chk(dalloc(&s->verts, 3 * (size_t)s->nv)); chk(dalloc(&s->faces, 3 * (size_t)n));
  chk(dalloc(&s->params, 2 * (size_t)n * s->ntex));
  chk(dalloc(&s->tri, 3 * (size_t)n)); chk(dalloc(&s->nodes, 4 * (size_t)std::max(n - 1, 1)));
  chk(dalloc(&s->parent, 2 * (size_t)n)); chk(dalloc(&s->flags, (size_t)std::max(n - 1, 1)));
  chk(dalloc(&s->keys, (size_t)n)); chk(dalloc(&s->keys2, (size_t)n)); chk(dalloc(&s->ids, (size_t)n));
  chk(dalloc(&s->ids2, (size_t)n)); chk(dalloc(&s->hist, 256 * (size_t)s->sort_blocks)); chk(dalloc(&s->bounds, 6));
  chk(dalloc(&s->nodes4, 7 * (size_t)std::max(n - 1, 1))); chk(dalloc(&s->src4, 4 * (size_t)std::max(n - 1, 1)));
  chk(dalloc(&s->q4, 4 * (size_t)n)); chk(dalloc(&s->c4, 2));
  chk(dalloc(&s->lights, 2 * (size_t)std::max(s->nl, 1))); chk(dalloc(&s->edge_v, ev.size()));
  chk(dalloc(&s->edge_f, ef.size())); chk(dalloc(&s->d_args, 1)); chk(dalloc(&s->d_err, 1));
  chk(dalloc(&s->mstat, 1));
  {
    // edge hierarchy: at most 2^14 leaf blocks of at least 4 edges
    int nE = s->n_edges;
    s->et_G = std::max(4, (nE + (1 << 14) - 1) >> 14);
    s->et_nleaf = (nE + s->et_G - 1) / s->et_G;
    s->et_L = 0;
    while ((1 << s->et_L) < s->et_nleaf) ++s->et_L;
    chk(dalloc(&s->et_lo, (size_t)2 << s->et_L)); chk(dalloc(&s->et_hi, (size_t)2 << s->et_L));
    chk(dalloc(&s->et_cn, (size_t)2 << s->et_L));
  }
  std::vector<int> vfs, vfl;
  if (s->smooth) {
    // faces around each vertex, in face order (CSR)
    vfs.assign((size_t)s->nv + 1, 0);
    for (int v : hf) ++vfs[(size_t)v + 1];
    for (int v = 0; v < s->nv; ++v) vfs[(size_t)v + 1] += vfs[v];
    vfl.resize(hf.size());
    std::vector<int> cur(vfs.begin(), vfs.end() - 1);
    for (int f = 0; f < n; ++f)
      for (int k = 0; k < 3; ++k) vfl[(size_t)cur[hf[3 * (size_t)f + k]]++] = f;
    chk(dalloc(&s->vnrm, (size_t)s->nv)); chk(dalloc(&s->vf_start, vfs.size())); chk(dalloc(&s->vf_list, vfl.size()));
    chk(dalloc(&s->dN, 3 * (size_t)s->nv));
  }
  if (d->env) { chk(dalloc(&s->env_tex, etex.size())); chk(dalloc(&s->env_alias, etab.size())); }
  if (e != cudaSuccess) { destroy(s); cudaGetLastError(); return fail(ST_ERR_OOM, "scene buffers"); }
  std::vector<float4> hl(2 * (size_t)std::max(s->nl, 1), make_float4(0, 0, 0, 0));
  for (int j = 0; j < s->nl; ++j) {
    const st_point_light& L = d->point_lights[j];
    s->host_lights.push_back(L);
    hl[2 * j] = make_float4(L.pos[0], L.pos[1], L.pos[2], 0.0f);
    hl[2 * j + 1] = make_float4(L.intensity[0], L.intensity[1], L.intensity[2], 0.0f);
  }
  chk(copy_async(s->verts, d->vertices, 3 * sizeof(float) * s->nv, cudaMemcpyDeviceToDevice, st));
  chk(copy_async(s->faces, d->faces, 3 * sizeof(int) * n, cudaMemcpyDeviceToDevice, st));
  {
    int nt = n * s->ntex;
    k_params_in<<<(nt + 255) / 256, 256, 0, st>>>(d->face_params, s->params, nt, s->np);
  }
  chk(copy_async(s->lights, hl.data(), hl.size() * sizeof(float4), cudaMemcpyHostToDevice, st));
  chk(copy_async(s->edge_v, ev.data(), ev.size() * sizeof(int2), cudaMemcpyHostToDevice, st));
  chk(copy_async(s->edge_f, ef.data(), ef.size() * sizeof(int2), cudaMemcpyHostToDevice, st));
  chk(cudaMemsetAsync(s->d_err, 0, sizeof(int), st));
  if (s->smooth) {
    chk(copy_async(s->vf_start, vfs.data(), vfs.size() * sizeof(int), cudaMemcpyHostToDevice, st));
    chk(copy_async(s->vf_list, vfl.data(), vfl.size() * sizeof(int), cudaMemcpyHostToDevice, st));
  }
  if (d->env) {
    chk(copy_async(s->env_tex, etex.data(), etex.size() * sizeof(float4), cudaMemcpyHostToDevice, st));
    chk(copy_async(s->env_alias, etab.data(), etab.size() * sizeof(float2), cudaMemcpyHostToDevice, st));
    s->env.w = d->env->width;
    s->env.h = d->env->height;
    s->env.tex = s->env_tex;
    s->env.alias = s->env_alias;
    s->env.pdf_scale = (float)((double)d->env->width * d->env->height / (2.0 * 3.14159265358979323846 * 3.14159265358979323846));
  }
  chk(cudaStreamCreateWithFlags(&s->cap_stream, cudaStreamNonBlocking));
  for (auto& a : s->aux_stream) chk(cudaStreamCreateWithFlags(&a, cudaStreamNonBlocking));
  if (e == cudaSuccess) e = s->builder == ST_BVH_LBVH ? bvh_build(s, st) : bvh_build_ploc(s, st);
  if (e == cudaSuccess) e = bvh_collapse(s, st);
  if (e == cudaSuccess) e = mesh_stat(s, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) { destroy(s); return cuda_fail(e, "scene create"); }
  *out = s;
  return ST_OK;
}

st_status st_scene_destroy(st_scene* s) {
  destroy(s);
  return ST_OK;
}

static st_status update_vertices(st_scene* s, const float* v, void* stream, bool rebuild) {
  if (!s || !v) return fail(ST_ERR_INVALID_ARG, "NULL argument");
  s->geom_version++;   // the primary-visibility bins and point-light lists are rebuilt by the next call
  cudaStream_t st = (cudaStream_t)stream;
  ST_CUDA(copy_async(s->verts, v, 3 * sizeof(float) * s->nv, cudaMemcpyDeviceToDevice, st));
  cudaError_t e = !rebuild ? bvh_refit(s, st) : s->builder == ST_BVH_LBVH ? bvh_build(s, st) : bvh_build_ploc(s, st);
  if (e == cudaSuccess && rebuild) e = bvh_collapse(s, st);
  if (e == cudaSuccess) e = mesh_stat(s, st);
  if (e != cudaSuccess) return cuda_fail(e, rebuild ? "rebuild" : "refit");
  return ST_OK;
}

st_status st_refit(st_scene* s, const float* v, void* stream) { return update_vertices(s, v, stream, false); }
st_status st_rebuild(st_scene* s, const float* v, void* stream) { return update_vertices(s, v, stream, true); }

st_status st_set_face_params(st_scene* s, const float* p, void* stream) {
  if (!s || !p) return fail(ST_ERR_INVALID_ARG, "NULL argument");
  int nt = s->nf * s->ntex;
  k_params_in<<<(nt + 255) / 256, 256, 0, (cudaStream_t)stream>>>(p, s->params, nt, s->np);
  ST_CUDA(cudaGetLastError());
  return ST_OK;
}

st_status st_render(st_scene* s, const st_view* views, int n_views, int default_spp, int max_bounces,
                    unsigned long long seed, const st_render_opts* opts, float* out_image, void* stream) {
  Range range("st_render");
  if (!s || !out_image) return fail(ST_ERR_INVALID_ARG, "NULL argument");
  Plan p;
  st_status r = plan_call(s, views, n_views, default_spp, max_bounces, opts, 0, false, p);
  if (r != ST_OK) return r;
  CallArgs a{(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32), out_image, nullptr, nullptr, nullptr,
             p.o.path_signatures};
  return run_call(s, p, a, (cudaStream_t)stream);
}

st_status st_render_backward(st_scene* s, const st_view* views, int n_views, int default_spp, int max_bounces,
                             unsigned long long seed, const st_render_opts* opts, const float* dLdI, float* dV,
                             float* dF, void* stream) {
  Range range("st_render_backward");
  if (!s || !dLdI) return fail(ST_ERR_INVALID_ARG, "NULL argument");
  st_render_opts o = opts ? *opts : default_opts();
  if (o.edge_term && !dV) return fail(ST_ERR_INVALID_ARG, "edge term needs d_vertices");
  if (!dV && !dF) return fail(ST_ERR_INVALID_ARG, "no gradient requested");
  Plan p;
  st_status r = plan_call(s, views, n_views, default_spp, max_bounces, &o, 1, true, p);
  if (r != ST_OK) return r;
  CallArgs a{(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32), nullptr, dLdI, dV, dF, nullptr};
  return run_call(s, p, a, (cudaStream_t)stream);
}

st_status st_trace_closest(st_scene* s, const float* rays, int n, int exclude, int* out_tri, float* out_t,
                           void* stream) {
  if (!s || (n > 0 && (!rays || !out_tri || !out_t)) || n < 0) return fail(ST_ERR_INVALID_ARG, "bad arguments");
  if (n == 0) return ST_OK;
  k_trace_rays<<<(n + EXT_BLOCK - 1) / EXT_BLOCK, EXT_BLOCK, 0, (cudaStream_t)stream>>>(
      s->nodes4, s->tri, s->nf, s->n4, (const float4*)rays, n, exclude, out_tri, out_t, s->d_err);
  ST_CUDA(cudaGetLastError());
  return ST_OK;
}

st_status st_get_stats(st_scene* s, st_stats* out) {
  if (!s || !out) return fail(ST_ERR_INVALID_ARG, "NULL argument");
  ST_CUDA(cudaDeviceSynchronize());
  st_stats r;
  std::memset(&r, 0, sizeof(r));
  unsigned long long h[STAT_SIZE] = {0};
  if (s->eng.stat) ST_CUDA(copy_sync(h, s->eng.stat, sizeof(h), cudaMemcpyDeviceToHost));
  for (auto& e : s->eng2) {
    // an overlapped call counts in every engine (all are zeroed at the start of every call)
    if (!e.stat) continue;
    unsigned long long h2[STAT_SIZE] = {0};
    ST_CUDA(copy_sync(h2, e.stat, sizeof(h2), cudaMemcpyDeviceToHost));
    for (int i = 0; i < STAT_SIZE; ++i) h[i] += h2[i];
  }
  int err = 0;
  ST_CUDA(copy_sync(&err, s->d_err, sizeof(int), cudaMemcpyDeviceToHost));
  r.paths = (long long)h[STAT_PATHS];
  r.extension_rays = (long long)h[STAT_EXT];
  r.shadow_rays = (long long)h[STAT_SHADOW];
  r.node_visits = (long long)h[STAT_VISITS];
  r.tri_tests = (long long)h[STAT_TESTS];
  r.secondary_samples = (long long)h[STAT_SEC];
  r.shadow_node_visits = (long long)h[STAT_SH_VISITS];
  r.shadow_tri_tests = (long long)h[STAT_SH_TESTS];
  r.edge_samples = s->last_edge_samples;
  auto timed = [&](int k) {
    double ms = 0;
    for (int i = 0; i < s->ev_used[k]; ++i) {
      float x = 0;
      cudaEventElapsedTime(&x, s->ev[k][i].first, s->ev[k][i].second);
      ms += x;
    }
    return ms;
  };
  r.extend_launches = s->ev_used[0];
  r.extend_ms = timed(0);
  r.shadow_launches = s->ev_used[1];
  r.shadow_ms = timed(1);
  r.busy_ms = timed(2);
  r.host_syncs = s->host_syncs;
  r.device_error = err;
  r.bvh_nodes = std::max(s->nf - 1, 0);
  r.bvh4_nodes = s->n4;
  r.scratch_bytes = s->eng.bytes;
  for (auto& e : s->eng2) r.scratch_bytes += e.bytes;
  r.kernel_launches = s->launches;
  *out = r;
  return ST_OK;
}

st_status st_debug_bvh(st_scene* s, float* nodes, int* leaf_faces) {
  if (!s || !nodes || !leaf_faces) return fail(ST_ERR_INVALID_ARG, "NULL argument");
  ST_CUDA(cudaDeviceSynchronize());
  if (s->nf > 1) ST_CUDA(cudaMemcpy(nodes, s->nodes, sizeof(float4) * 4 * (s->nf - 1), cudaMemcpyDeviceToHost));
  ST_CUDA(cudaMemcpy(leaf_faces, s->ids, sizeof(int) * s->nf, cudaMemcpyDeviceToHost));
  return ST_OK;
}

// Measurement utility (not part of the path trace): read bandwidth of a buffer
// that stays resident in L2, so rooflines of L2-resident kernels (the BVH
// traversal) have a measured denominator beside the HBM copy bandwidth.
__global__ void k_l2_read(const float4* __restrict__ p, long long n4, int passes, float* out) {
  float4 acc = make_float4(0, 0, 0, 0);
  for (int r = 0; r < passes; ++r)
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n4; i += (long long)gridDim.x * blockDim.x) {
      float4 v = __ldcg(p + i);
      acc.x += v.x; acc.y += v.y; acc.z += v.z; acc.w += v.w;
    }
  float sum = acc.x + acc.y + acc.z + acc.w;
  if (sum == -1.0f) out[blockIdx.x] = sum;   // keeps the loads; the buffer holds zeros, so this never stores
}

st_status st_measure_l2_read(long long bytes, int passes, void* stream, double* gbs) {
  if (bytes < (1 << 20) || passes < 1 || !gbs) return fail(ST_ERR_INVALID_ARG, "bad arguments");
  cudaStream_t st = (cudaStream_t)stream;
  long long n4 = bytes / 16;
  float4* buf = nullptr;
  float* out = nullptr;
  cudaEvent_t a = nullptr, b = nullptr;
  int dev = 0, sm = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sm, cudaDevAttrMultiProcessorCount, dev);
  int grid = sm * 4;
  cudaError_t e = cudaMalloc((void**)&buf, n4 * 16);
  if (e == cudaSuccess) e = cudaMalloc((void**)&out, sizeof(float) * grid);
  if (e == cudaSuccess) e = cudaMemsetAsync(buf, 0, n4 * 16, st);
  if (e == cudaSuccess) e = cudaEventCreate(&a);
  if (e == cudaSuccess) e = cudaEventCreate(&b);
  if (e == cudaSuccess) {
    k_l2_read<<<grid, 512, 0, st>>>(buf, n4, 2, out);   // warm: the buffer becomes L2 resident
    cudaEventRecord(a, st);
    k_l2_read<<<grid, 512, 0, st>>>(buf, n4, passes, out);
    cudaEventRecord(b, st);
    e = cudaEventSynchronize(b);
  }
  float ms = 0;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  if (buf) cudaFree(buf);
  if (out) cudaFree(out);
  if (e != cudaSuccess) return cuda_fail(e, "st_measure_l2_read");
  *gbs = (double)n4 * 16.0 * passes / (ms / 1000.0) / 1e9;
  return ST_OK;
}

}  // extern "C"
