// C ABI of the hz library: plan creation (1D operators, eigen-decompositions,
// device tables, z factors), the solve orchestration of steps 1-7 of Sec. 2, the
// mixed-precision refinement, adjoint and layer gradient, batched graph launches, the
// autotuners and the GMRES of the locally perturbed medium.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <complex>
#include <cstring>
#include <memory>
#include <new>
#include <vector>

#include <nvtx3/nvToolsExt.h>   // header-only; the ranges cost nothing unless a profiler is attached

#include "hz_internal.h"

using hz::cd;

namespace hz {
namespace {
std::atomic<long long> g_launches{0};
}
void count_launch(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
long long launch_count() { return g_launches.load(std::memory_order_relaxed); }
}  // namespace hz

namespace {

constexpr int kTileN = 16;   // output columns per transform tile (matches hz_xform.cu)

// ---------------------------------------------------------------------------
// Host-side axis data
// ---------------------------------------------------------------------------
struct AxisPlan {
  int n = 0, nb = 1;
  std::vector<cd> h, mh, kd, ko;             // steps, dual lengths, stiffness (diag, off)
  std::vector<int> bstart, bsize, iface;
  std::vector<std::vector<cd>> blam, bW;     // per block eigenpairs (W row-major [node][mode])
  std::vector<int> breal;
  std::vector<int> bsym;                     // uniform block: sine pairs, symmetric modes first
  std::vector<cd> glam, gW;                  // whole-axis eigenpairs (when the plan needs them)
  int greal = 0, gsym = 0;
  double eig_res = 0.0;
};

// Device tables of one axis.
struct AxisDev {
  hz::XformSet fwd, inv, gfwd, ginv;
  hz::TCSet tfwd, tinv;                          // tensor-core copies of fwd / inv (mixed path)
  double2 *lam_b = nullptr, *lam_g = nullptr;    // eigenvalue per position (block / global)
  signed char* skip = nullptr;                   // interface flags
  int* ifc = nullptr;                            // interface node indices
  double2 *m = nullptr, *im = nullptr, *ih = nullptr;
  double2* edge_coef = nullptr;  int2* edge_rng = nullptr;   // 2 nI slots (step 3)
  double2* gcoef = nullptr;      int2* grng = nullptr;       // nI slots (step 5), Wg[p][:]
  int *gl = nullptr, *gr = nullptr;                          // pass B interface indices
  double2 *cl = nullptr, *cr = nullptr;                      // pass B coefficients
  float2 *edge_coef32 = nullptr, *gcoef32 = nullptr;         // FP32 copies (mixed path)
  float2 *cl32 = nullptr, *cr32 = nullptr;
  double2* ks = nullptr;                                     // stencil rows / mhat
  signed char* kreal = nullptr;                              // off-diagonals of row real
  bool edge_real = false, g_real = false, lr_real = false;   // edge_coef, gcoef, cl/cr all real
};

struct Workspace {
  int cap = 0;                       // RHS capacity
  double2 *FT = nullptr, *G = nullptr, *V = nullptr;
  double2 *cX = nullptr, *vX = nullptr, *cY = nullptr, *vY = nullptr;
  double2 *rX = nullptr, *rY = nullptr, *aX = nullptr, *bY = nullptr;
  double2 *cg = nullptr, *dg = nullptr, *wX = nullptr, *wY = nullptr;
  double2 *alX = nullptr, *alY = nullptr;
  double2 *RHO = nullptr, *F2 = nullptr;           // residual / input copy (mixed, adjoint, host)
  double2 *HU = nullptr;                           // output staging for host solves
  double* partial = nullptr; double* norms = nullptr;
  double2* gpart = nullptr; double2* Gl = nullptr;
  int rho_cap = 0, f2_cap = 0, hu_cap = 0;
};

}  // namespace

struct hz_plan_s {
  int nx = 0, ny = 0, nz = 0, nlayers = 0;
  int device = 0;                    // the device current at plan creation (owns tables and stream)
  hz_options opts{};
  cudaStream_t st = nullptr;
  AxisPlan ax, ay;
  std::vector<cd> hz, k2base;
  std::vector<double> sig_layer;
  std::vector<int> z_begin;
  double omega = 1.0;
  bool need_global = false;
  bool use_tc = true;                // mixed path: bulk transforms on the tensor cores
  bool tc_ok = true;                 // the tensor-core tables have their TMA tensor maps
  bool fast_sine = true;             // FP64 path: uniform blocks through the FFT-based sine transform
  bool fast_sine32 = false;          // mixed path: the same in FP32 instead of the tensor cores
  bool tc_real = true;               // mixed path: real tables through the real-table kernel
  bool has_real_tc = false;          // some block has a real table
  bool has_dst = false;              // some block has a fast sine transform
  int zs_rb = 0;                     // z sweep variant (hz_plan_set_z_sweep; 0 automatic; autotuned)
  int xf_tile = 0;                   // data rows per CTA of the dense transforms: 16, 64, 0 by launch size (autotuned)
  int sms = 0;                       // SM count of the plan's device
  // second stream for the y-side interface work (runs beside the x side)
  cudaStream_t side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  cudaStream_t cst = nullptr;                  // host -> device copies overlapped with solves
  cudaStream_t cst2 = nullptr;                 // device -> host copies overlapped with solves
  cudaEvent_t ev_in[8] = {};                   // upload of chunk c done
  int real_cm = 1;
  AxisDev dx, dy;
  // z tables
  double2 *tzd = nullptr, *szs = nullptr, *mz = nullptr, *imz = nullptr, *coff = nullptr;
  double2 *cm_b = nullptr, *cm_g = nullptr, *tzs = nullptr;
  double* sig = nullptr;
  // residual-stencil tables
  double2* cxy = nullptr;
  double *w2xy = nullptr, *w2z = nullptr;
  signed char* rz = nullptr;
  int* zb = nullptr;
  // factors
  double2 *Pb = nullptr, *Qb = nullptr, *Pg = nullptr, *Qg = nullptr;
  int* status = nullptr;
  unsigned long long* minpiv = nullptr;
  Workspace ws;
  std::vector<void*> allocs;
  long long bytes = 0;
  hz_info info{};
  // stage timers
  bool timing = false;
  double stage_ms[HZ_NSTAGES] = {};
  long long stage_launches[HZ_NSTAGES] = {};
  std::vector<cudaEvent_t> ev_pool;
  struct Rec { int stage; cudaEvent_t a, b; long long launches; };
  std::vector<Rec> recs;
  size_t ev_used = 0;
};

namespace {

// ---------------------------------------------------------------------------
// helpers
// ---------------------------------------------------------------------------
struct Fail {
  hz_status s;
};

void ck(cudaError_t e) {
  if (e == cudaErrorMemoryAllocation) throw Fail{HZ_ERR_OOM};
  if (e != cudaSuccess) throw Fail{HZ_ERR_CUDA};
}

// A named NVTX range for profilers (host timeline; the launches inside it correlate).
class NvtxRange {
 public:
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

const char* const kStageNames[HZ_NSTAGES] = {
    "hz step 1: forward x/y transforms", "hz step 2: block z solves",
    "hz step 3: v next to the interfaces", "hz step 4: interface residual",
    "hz step 5: global interface solve", "hz step 6: boundary terms and block z solves",
    "hz step 7: inverse x/y transforms", "hz step 7: u on the interfaces",
    "hz residual / refinement"};

// Records CUDA events around a stage when the plan's stage timers are on, and marks the
// stage as an NVTX range.
class Stage {
 public:
  Stage(hz_plan_t p, cudaStream_t st, int stage)
      : range_(kStageNames[stage]), p_(p), st_(st), stage_(stage), l0_(hz::launch_count()) {
    if (p_->timing) a_ = next_event(), ck(cudaEventRecord(a_, st_));
  }
  ~Stage() {
    if (p_->timing) {
      cudaEvent_t b = next_event();
      cudaEventRecord(b, st_);
      p_->recs.push_back({stage_, a_, b, hz::launch_count() - l0_});
    }
  }

 private:
  cudaEvent_t next_event() {
    if (p_->ev_used == p_->ev_pool.size()) {
      cudaEvent_t e;
      ck(cudaEventCreate(&e));
      p_->ev_pool.push_back(e);
    }
    return p_->ev_pool[p_->ev_used++];
  }
  NvtxRange range_;
  hz_plan_t p_;
  cudaStream_t st_;
  int stage_;
  long long l0_;
  cudaEvent_t a_ = nullptr;
};

// After the stream is synchronised: fold the recorded event pairs into the totals.
void collect_stages(hz_plan_t p) {
  for (const auto& r : p->recs) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) p->stage_ms[r.stage] += ms;
    p->stage_launches[r.stage] += r.launches;
  }
  p->recs.clear();
  p->ev_used = 0;
}

template <typename T>
T* dalloc(hz_plan_t p, size_t count) {
  if (count == 0) count = 1;
  void* ptr = nullptr;
  ck(cudaMalloc(&ptr, count * sizeof(T)));
  ck(cudaMemsetAsync(ptr, 0, count * sizeof(T), p->st));
  p->allocs.push_back(ptr);
  p->bytes += (long long)(count * sizeof(T));
  return static_cast<T*>(ptr);
}

void dfree(hz_plan_t p, void* ptr) {
  if (!ptr) return;
  auto it = std::find(p->allocs.begin(), p->allocs.end(), ptr);
  if (it != p->allocs.end()) p->allocs.erase(it);
  cudaFree(ptr);
}

template <typename T>
T* upload(hz_plan_t p, const std::vector<T>& v) {
  T* d = dalloc<T>(p, v.size());
  if (!v.empty()) ck(cudaMemcpyAsync(d, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, p->st));
  return d;
}

double2* upload_c(hz_plan_t p, const std::vector<cd>& v) {
  std::vector<double2> t(v.size());
  for (size_t i = 0; i < v.size(); ++i) t[i] = make_double2(v[i].real(), v[i].imag());
  return upload(p, t);
}

float2* upload_c32(hz_plan_t p, const std::vector<cd>& v) {
  std::vector<float2> t(v.size());
  for (size_t i = 0; i < v.size(); ++i) t[i] = make_float2((float)v[i].real(), (float)v[i].imag());
  return upload(p, t);
}

bool finite(cd z) { return std::isfinite(z.real()) && std::isfinite(z.imag()); }

// ---------------------------------------------------------------------------
// Plan construction
// ---------------------------------------------------------------------------
// Automatic block count for an axis of n nodes.  FP64 operations per unknown and solve,
// per axis: the dense block transforms of steps 1 and 7 cost about 12 n / B (two
// transforms, 3 FMA per complex multiply-add, blocks n / B wide); the interface steps
// (short whole-axis transforms, the rank-|I| right-hand sides and contractions of steps
// 5 and 6) about 28 (B - 1).  The minimum is at B = sqrt(3 n / 7) ~ 0.65 sqrt(n), the
// sqrt(N) partition of the cost estimate in Sec. 2; blocks stay at least 16 nodes wide
// (one transform column tile).  The mixed path runs the block transforms on tensor cores
// at memory speed, so there fewer, wider blocks win: about 80 nodes each.
int auto_blocks(int n, bool mixed) {
  int b = mixed ? (int)std::lround(n / 80.0) : (int)std::lround(std::sqrt(3.0 * n / 7.0));
  b = std::min(b, n / 16);
  return std::max(b, 1);
}

// True when the sz + 1 steps h[s .. s + sz] that touch the nodes s .. s + sz - 1 are all
// equal, real and positive: that block's pencil has the closed-form sine pairs.
bool uniform_steps(const std::vector<cd>& h, int s, int sz, double* hu) {
  const cd h0 = h[s];
  if (h0.imag() != 0.0 || !(h0.real() > 0.0)) return false;
  for (int i = s; i <= s + sz; ++i)
    if (h[i] != h0) return false;
  *hu = h0.real();
  return true;
}

hz_status build_axis(AxisPlan& A, int n, const hz_c128* h, int nb, const int* ifc) {
  A.n = n;
  A.nb = nb;
  A.h.resize(n + 1);
  for (int i = 0; i <= n; ++i) {
    A.h[i] = cd(h[i].re, h[i].im);
    if (!finite(A.h[i]) || std::abs(A.h[i]) == 0.0) return HZ_ERR_ARG;
  }
  A.mh.resize(n);
  A.kd.resize(n);
  A.ko.resize(std::max(n - 1, 0));
  for (int i = 0; i < n; ++i) {
    A.mh[i] = 0.5 * (A.h[i] + A.h[i + 1]);
    A.kd[i] = 1.0 / A.h[i] + 1.0 / A.h[i + 1];
    if (i + 1 < n) A.ko[i] = -1.0 / A.h[i + 1];
  }
  A.iface.clear();
  for (int b = 1; b < nb; ++b) A.iface.push_back(ifc ? ifc[b - 1] : (b * (n + 1)) / nb - 1);
  int prev = -1;
  A.bstart.clear();
  A.bsize.clear();
  for (int b = 0; b < nb; ++b) {
    const int end = (b < nb - 1) ? A.iface[b] : n;
    const int size = end - prev - 1;
    if (size < 1) return HZ_ERR_ARG;
    A.bstart.push_back(prev + 1);
    A.bsize.push_back(size);
    prev = end;
  }
  A.blam.assign(nb, {});
  A.bW.assign(nb, {});
  A.breal.assign(nb, 1);
  A.bsym.assign(nb, 0);
  A.eig_res = 0.0;
  for (int b = 0; b < nb; ++b) {
    const int s = A.bstart[b], sz = A.bsize[b];
    double res = 0.0;
    double hu = 0.0;
    A.bsym[b] = uniform_steps(A.h, s, sz, &hu) ? 1 : 0;
    const bool ok = A.bsym[b]
                        ? hz::sine_eig(sz, hu, &A.kd[s], sz > 1 ? &A.ko[s] : nullptr, &A.mh[s], A.blam[b],
                                       A.bW[b], &res)
                        : hz::tridiag_eig(sz, &A.kd[s], sz > 1 ? &A.ko[s] : nullptr, &A.mh[s], A.blam[b],
                                          A.bW[b], &res);
    if (!ok) return HZ_ERR_EIG;
    A.eig_res = std::max(A.eig_res, res);
    for (const cd& w : A.bW[b])
      if (w.imag() != 0.0) { A.breal[b] = 0; break; }
  }
  return HZ_OK;
}

hz_status build_global(AxisPlan& A) {
  if (A.nb == 1) {
    A.glam = A.blam[0];
    A.gW = A.bW[0];
    A.greal = A.breal[0];
    A.gsym = A.bsym[0];
    return HZ_OK;
  }
  double res = 0.0;
  double hu = 0.0;
  A.gsym = uniform_steps(A.h, 0, A.n, &hu) ? 1 : 0;
  const bool ok = A.gsym
                      ? hz::sine_eig(A.n, hu, A.kd.data(), A.ko.data(), A.mh.data(), A.glam, A.gW, &res)
                      : hz::tridiag_eig(A.n, A.kd.data(), A.ko.data(), A.mh.data(), A.glam, A.gW, &res);
  if (!ok) return HZ_ERR_EIG;
  A.eig_res = std::max(A.eig_res, res);
  A.greal = 1;
  for (const cd& w : A.gW)
    if (w.imag() != 0.0) { A.greal = 0; break; }
  return HZ_OK;
}

// Pack a block-diagonal transform: tab(b)[a][c] = get(b, a, c).
template <typename Get>
// sym[b] marks a uniform block (sine pairs, symmetric modes first); dir = 1 for a forward
// table (rows = nodes), 2 for an inverse table (rows = modes).  The table is stored whole
// either way; symmetric blocks read half of it (see the row-transform kernels).
// fast[b]: block b takes the fast sine transform (a uniform block, dst_supported(size[b])).
void make_xform(hz_plan_t p, hz::XformSet& xs, int ncols, const std::vector<int>& start,
                const std::vector<int>& size, const std::vector<int>& real, const std::vector<int>& sym,
                int dir, const std::vector<char>& fastb, Get get) {
  xs.ncols = ncols;
  xs.nblocks = (int)start.size();
  std::vector<hz::XBlock> blocks;
  std::vector<hz::XTile> tiles;
  std::vector<double> t64;
  std::vector<float> t32;
  for (int b = 0; b < xs.nblocks; ++b) {
    const int n = size[b];
    hz::XBlock xb{};
    xb.start = start[b];
    xb.size = n;
    xb.real = real[b];
    xb.sym = (sym[b] && real[b]) ? dir : 0;
    xb.ns = (n + 1) / 2;
    xb.toff = (long long)t64.size();
    xb.toff32 = (long long)t32.size();
    const size_t nn = (size_t)n * n;
    if (real[b]) {
      t64.resize(t64.size() + nn);
      t32.resize(t32.size() + nn);
      for (int a = 0; a < n; ++a)
        for (int c = 0; c < n; ++c) {
          const double v = get(b, a, c).real();
          t64[xb.toff + (size_t)a * n + c] = v;
          t32[xb.toff32 + (size_t)a * n + c] = (float)v;
        }
    } else {
      t64.resize(t64.size() + 3 * nn);
      t32.resize(t32.size() + 2 * nn);
      for (int a = 0; a < n; ++a)
        for (int c = 0; c < n; ++c) {
          const cd v = get(b, a, c);
          const size_t o = (size_t)a * n + c;
          t64[xb.toff + o] = v.real();
          t64[xb.toff + nn + o] = v.imag() - v.real();
          t64[xb.toff + 2 * nn + o] = v.real() + v.imag();
          t32[xb.toff32 + o] = (float)v.real();
          t32[xb.toff32 + nn + o] = (float)v.imag();
        }
    }
    blocks.push_back(xb);
    // inverse tables of symmetric blocks produce two nodes per column: tiles cover the first ns
    const int ncov = xb.sym == 2 ? xb.ns : n;
    for (int c0 = 0; c0 < ncov; c0 += kTileN) tiles.push_back(hz::XTile{b, c0, std::min(kTileN, ncov - c0), 0});
  }
  xs.ntiles = (int)tiles.size();
  xs.h_blocks = blocks;
  xs.d_blocks = upload(p, blocks);
  xs.d_tiles = upload(p, tiles);
  xs.d_tab = upload(p, t64);
  xs.d_tab32 = upload(p, t32);
  // FP64 fast sine transforms of the uniform blocks: the table must be S sin(pi j m / N)
  // (rows j = nodes, columns m = modes in the symmetric-first order, or the transpose)
  std::vector<hz::DstBlock> dblk;
  std::vector<int> didx;
  std::vector<double> dcoef;
  std::vector<double2> dtw;
  std::vector<char> fast(xs.nblocks, 0);
  const double pi = 3.14159265358979323846;
  for (int b = 0; b < xs.nblocks; ++b) {
    const hz::XBlock& xb = blocks[b];
    if (!fastb[b]) continue;
    if (!xb.sym) throw Fail{HZ_ERR_EIG};
    const int n = xb.size, N = n + 1, ns = (n + 1) / 2;
    auto mode = [&](int c) { return c < ns ? 2 * c + 1 : 2 * (c - ns) + 2; };
    const double S = get(b, 0, 0).real() / std::sin(pi / N);
    double dev = 0.0;
    for (int a = 0; a < n; ++a)
      for (int c = 0; c < n; ++c) {
        const long long jm = (dir == 1) ? (long long)(a + 1) * mode(c) : (long long)mode(a) * (c + 1);
        const double ref = S * std::sin((double)(jm % (2 * N)) * pi / N);
        dev = std::max(dev, std::abs(get(b, a, c) - cd(ref)));
      }
    // the closed-form sine table and the fast transform must agree (the tensor-core tile subset
    // already leaves this block out)
    if (!(dev <= 1e-13 * std::abs(S)) || !hz::dst_plan_block(n, xb.start, dir, S, dblk, didx, dcoef, dtw))
      throw Fail{HZ_ERR_EIG};
    fast[b] = 1;
    xs.dst.nmax = std::max(xs.dst.nmax, N);
  }
  std::vector<hz::XTile> tiles64;
  for (const auto& t : tiles)
    if (!fast[t.blk]) tiles64.push_back(t);
  xs.ntiles64 = (int)tiles64.size();
  xs.d_tiles64 = upload(p, tiles64);
  xs.dst.nblk = (int)dblk.size();
  if (xs.dst.nblk) {
    xs.dst.d_blk = upload(p, dblk);
    xs.dst.d_idx = upload(p, didx);
    xs.dst.d_coef = upload(p, dcoef);
    xs.dst.d_tw = upload(p, dtw);
    std::vector<float> c32(dcoef.begin(), dcoef.end());
    std::vector<float2> t32(dtw.size());
    for (size_t i = 0; i < dtw.size(); ++i) t32[i] = make_float2((float)dtw[i].x, (float)dtw[i].y);
    xs.dst.d_coef32 = upload(p, c32);
    xs.dst.d_tw32 = upload(p, t32);
    p->has_dst = true;
  }
}

// Tensor-core tables of a block-diagonal transform: tab(b)[a][c] = get(b, a, c).
template <typename Get>
void make_tc(hz_plan_t p, hz::TCSet& ts, int ncols, const std::vector<int>& start,
             const std::vector<int>& size, const std::vector<char>& fastb, Get get) {
  std::vector<float> tab;
  std::vector<hz::TCBlock> blocks(start.size());
  std::vector<hz::TCTile> tiles, rtiles;
  for (size_t b = 0; b < start.size(); ++b) {
    const int n = size[b];
    std::vector<cd> B((size_t)n * n);
    bool real = true;
    for (int a = 0; a < n; ++a)
      for (int c = 0; c < n; ++c) {
        B[(size_t)a * n + c] = get((int)b, a, c);
        if (B[(size_t)a * n + c].imag() != 0.0) real = false;
      }
    hz::tc_pack_block(B.data(), n, start[b], tab, blocks[b], tiles, (int)b, real ? &rtiles : nullptr);
  }
  ts.ncols = ncols;
  ts.d_blocks = upload(p, blocks);
  ts.d_tab = upload(p, tab);
  if (!rtiles.empty()) p->has_real_tc = true;
  // tile lists per variant v = fast + 2 real (see TCSet)
  for (int v = 0; v < 4; ++v) {
    const bool fast = v & 1, real = v & 2;
    std::vector<hz::TCTile> cl, rl;
    for (const auto& t : tiles)
      if (!(fast && fastb[t.blk]) && !(real && blocks[t.blk].npad_r > 0)) cl.push_back(t);
    if (real)
      for (const auto& t : rtiles)
        if (!(fast && fastb[t.blk])) rl.push_back(t);
    for (int k = 0; k < 2; ++k) {
      const std::vector<hz::TCTile>& lt = k ? rl : cl;
      hz::TCList& L = k ? ts.rl[v] : ts.cl[v];
      L.ntiles = (int)lt.size();
      if (lt.empty()) continue;
      for (const auto& t : lt) L.nt_max = std::max(L.nt_max, t.nt);
      L.d_tiles = upload(p, lt);
      std::vector<unsigned char> maps;
      if (p->tc_ok && hz::tc_encode_tmaps(ts.d_tab, blocks, lt, maps, k == 1)) L.d_tmaps = upload(p, maps);
      else p->use_tc = p->tc_ok = false;   // no tensor maps: the mixed path runs the SIMT FP32 transforms
    }
  }
}

void build_axis_dev(hz_plan_t p, const AxisPlan& A, AxisDev& D, bool need_global) {
  const int n = A.n, nI = (int)A.iface.size();
  // uniform blocks whose width suits the FFT take the fast sine transform (FP64 and mixed paths)
  std::vector<char> fastb(A.nb, 0);
  for (int b = 0; b < A.nb; ++b) fastb[b] = (A.bsym[b] && A.breal[b] && hz::dst_supported(A.bsize[b])) ? 1 : 0;
  make_tc(p, D.tfwd, n, A.bstart, A.bsize, fastb, [&](int b, int a, int c) {
    return A.mh[A.bstart[b] + a] * A.bW[b][(size_t)a * A.bsize[b] + c];
  });
  make_tc(p, D.tinv, n, A.bstart, A.bsize, fastb,
          [&](int b, int a, int c) { return A.bW[b][(size_t)c * A.bsize[b] + a]; });
  make_xform(p, D.fwd, n, A.bstart, A.bsize, A.breal, A.bsym, 1, fastb, [&](int b, int a, int c) {
    return A.mh[A.bstart[b] + a] * A.bW[b][(size_t)a * A.bsize[b] + c];
  });
  make_xform(p, D.inv, n, A.bstart, A.bsize, A.breal, A.bsym, 2, fastb,
             [&](int b, int a, int c) { return A.bW[b][(size_t)c * A.bsize[b] + a]; });
  std::vector<cd> lam_b(n, cd(0)), lam_g(n, cd(0));
  std::vector<signed char> skip(n, 0);
  for (int q : A.iface) skip[q] = 1;
  for (int b = 0; b < A.nb; ++b)
    for (int a = 0; a < A.bsize[b]; ++a) lam_b[A.bstart[b] + a] = A.blam[b][a];
  if (need_global) {
    std::vector<int> s0{0}, sn{n}, gr{A.greal}, gs{A.gsym};
    std::vector<char> gf{(char)((A.gsym && A.greal && hz::dst_supported(n)) ? 1 : 0)};
    make_xform(p, D.gfwd, n, s0, sn, gr, gs, 1, gf, [&](int, int a, int c) { return A.gW[(size_t)a * n + c]; });
    make_xform(p, D.ginv, n, s0, sn, gr, gs, 2, gf, [&](int, int a, int c) { return A.gW[(size_t)c * n + a]; });
    lam_g = A.glam;
  }
  D.lam_b = upload_c(p, lam_b);
  D.lam_g = upload_c(p, lam_g);
  D.skip = upload(p, skip);
  D.ifc = upload(p, A.iface);
  std::vector<cd> im(n), ih(n + 1);
  for (int i = 0; i < n; ++i) im[i] = 1.0 / A.mh[i];
  for (int i = 0; i <= n; ++i) ih[i] = 1.0 / A.h[i];
  D.m = upload_c(p, A.mh);
  D.im = upload_c(p, im);
  D.ih = upload_c(p, ih);
  // step 3 edge rows: slot 2q = last row of the block left of interface q, 2q+1 = first row right of it
  std::vector<cd> ecoef((size_t)std::max(2 * nI, 1) * n, cd(0));
  std::vector<int2> erng(std::max(2 * nI, 1), make_int2(0, 0));
  for (int q = 0; q < nI; ++q) {
    const int bl = q, br = q + 1;
    const int sl = A.bstart[bl], nl = A.bsize[bl], sr = A.bstart[br], nr = A.bsize[br];
    for (int l = 0; l < nl; ++l) ecoef[(size_t)(2 * q) * n + sl + l] = A.bW[bl][(size_t)(nl - 1) * nl + l];
    for (int l = 0; l < nr; ++l) ecoef[(size_t)(2 * q + 1) * n + sr + l] = A.bW[br][(size_t)0 * nr + l];
    erng[2 * q] = make_int2(sl, sl + nl);
    erng[2 * q + 1] = make_int2(sr, sr + nr);
  }
  auto all_real = [](const std::vector<cd>& v) {
    for (const cd& z : v)
      if (z.imag() != 0.0) return false;
    return true;
  };
  D.edge_real = all_real(ecoef);
  D.edge_coef = upload_c(p, ecoef);
  D.edge_coef32 = upload_c32(p, ecoef);
  D.edge_rng = upload(p, erng);
  // step 5: rows of the whole-axis W at the interfaces
  std::vector<cd> gcoef((size_t)std::max(nI, 1) * n, cd(0));
  std::vector<int2> grng(std::max(nI, 1), make_int2(0, n));
  if (need_global)
    for (int q = 0; q < nI; ++q)
      for (int l = 0; l < n; ++l) gcoef[(size_t)q * n + l] = A.gW[(size_t)A.iface[q] * n + l];
  D.g_real = all_real(gcoef);
  D.gcoef = upload_c(p, gcoef);
  D.gcoef32 = upload_c32(p, gcoef);
  D.grng = upload(p, grng);
  // step 6: boundary right-hand side coefficients W[e][l] / h across the interface
  std::vector<int> gl(n, -1), grr(n, -1);
  std::vector<cd> cl(n, cd(0)), cr(n, cd(0));
  for (int b = 0; b < A.nb; ++b) {
    const int s = A.bstart[b], nb = A.bsize[b];
    for (int l = 0; l < nb; ++l) {
      if (b > 0) {
        gl[s + l] = b - 1;
        cl[s + l] = A.bW[b][(size_t)0 * nb + l] / A.h[s];
      }
      if (b < A.nb - 1) {
        grr[s + l] = b;
        cr[s + l] = A.bW[b][(size_t)(nb - 1) * nb + l] / A.h[s + nb];
      }
    }
  }
  D.gl = upload(p, gl);
  D.gr = upload(p, grr);
  D.lr_real = all_real(cl) && all_real(cr);
  D.cl = upload_c(p, cl);
  D.cr = upload_c(p, cr);
  D.cl32 = upload_c32(p, cl);
  D.cr32 = upload_c32(p, cr);
  // stencil rows divided by hhat
  std::vector<cd> ks((size_t)3 * n, cd(0));
  for (int i = 0; i < n; ++i) {
    if (i > 0) ks[3 * i + 0] = A.ko[i - 1] / A.mh[i];
    ks[3 * i + 1] = A.kd[i] / A.mh[i];
    if (i + 1 < n) ks[3 * i + 2] = A.ko[i] / A.mh[i];
  }
  D.ks = upload_c(p, ks);
  std::vector<signed char> kreal(n);
  for (int i = 0; i < n; ++i) kreal[i] = (ks[3 * i].imag() == 0.0 && ks[3 * i + 2].imag() == 0.0) ? 1 : 0;
  D.kreal = upload(p, kreal);
}

// Residual-stencil tables that combine both horizontal axes.
void build_stencil_xy(hz_plan_t p) {
  const int nx = p->nx, ny = p->ny;
  std::vector<cd> cxy((size_t)nx * ny);
  std::vector<double> w2((size_t)nx * ny);
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i) {
      cxy[(size_t)j * nx + i] = p->ax.kd[i] / p->ax.mh[i] + p->ay.kd[j] / p->ay.mh[j];
      w2[(size_t)j * nx + i] = std::norm(p->ax.mh[i]) * std::norm(p->ay.mh[j]);
    }
  p->cxy = upload_c(p, cxy);
  p->w2xy = upload(p, w2);
}

// z coefficients for the current k^2 (base * omega^2) and the mode factors.
void build_z(hz_plan_t p) {
  const int nz = p->nz;
  std::vector<cd> k2n(nz);
  std::vector<double> sn(nz, 1.0);
  for (int L = 0; L < p->nlayers; ++L)
    for (int k = p->z_begin[L]; k < p->z_begin[L + 1]; ++k) {
      k2n[k] = p->k2base[L] * (p->omega * p->omega);
      if (!p->sig_layer.empty()) sn[k] = p->sig_layer[L];
    }
  std::vector<double> shalf(nz + 1);
  shalf[0] = sn[0];
  shalf[nz] = sn[nz - 1];
  for (int k = 1; k < nz; ++k) shalf[k] = 2.0 * sn[k - 1] * sn[k] / (sn[k - 1] + sn[k]);
  std::vector<cd> mz(nz), imz(nz), szs(nz), tzd(nz), coff(nz, cd(0)), cmb(nz, cd(0)), cmg(nz, cd(0));
  std::vector<cd> tzs((size_t)3 * nz, cd(0));
  p->real_cm = 1;
  for (int k = 0; k < nz; ++k) {
    mz[k] = 0.5 * (p->hz[k] + p->hz[k + 1]);
    imz[k] = 1.0 / mz[k];
    szs[k] = sn[k] * mz[k];
    tzd[k] = shalf[k] / p->hz[k] + shalf[k + 1] / p->hz[k + 1] - k2n[k] * mz[k];
    if (k > 0) {
      coff[k] = -shalf[k] / p->hz[k];
      cmb[k] = coff[k] / mz[k];
      cmg[k] = coff[k];
      if (cmb[k].imag() != 0.0 || cmg[k].imag() != 0.0) p->real_cm = 0;
    }
  }
  for (int k = 0; k < nz; ++k) {
    if (k > 0) tzs[3 * k + 0] = coff[k] / mz[k];
    tzs[3 * k + 1] = tzd[k] / mz[k];
    if (k + 1 < nz) tzs[3 * k + 2] = coff[k + 1] / mz[k];
  }
  auto put = [&](double2*& d, const std::vector<cd>& v) {
    if (!d) d = dalloc<double2>(p, v.size());
    std::vector<double2> t(v.size());
    for (size_t i = 0; i < v.size(); ++i) t[i] = make_double2(v[i].real(), v[i].imag());
    ck(cudaMemcpyAsync(d, t.data(), t.size() * sizeof(double2), cudaMemcpyHostToDevice, p->st));
    ck(cudaStreamSynchronize(p->st));
  };
  put(p->mz, mz);
  put(p->imz, imz);
  put(p->szs, szs);
  put(p->tzd, tzd);
  put(p->coff, coff);
  put(p->cm_b, cmb);
  put(p->cm_g, cmg);
  put(p->tzs, tzs);
  {
    std::vector<double> w2z(nz);
    std::vector<signed char> rz(nz);
    for (int k = 0; k < nz; ++k) {
      w2z[k] = std::norm(mz[k]);
      rz[k] = (tzs[3 * k].imag() == 0.0 && tzs[3 * k + 2].imag() == 0.0) ? 1 : 0;
    }
    if (!p->w2z) p->w2z = dalloc<double>(p, nz);
    if (!p->rz) p->rz = dalloc<signed char>(p, nz);
    ck(cudaMemcpyAsync(p->w2z, w2z.data(), nz * sizeof(double), cudaMemcpyHostToDevice, p->st));
    ck(cudaMemcpyAsync(p->rz, rz.data(), nz, cudaMemcpyHostToDevice, p->st));
    ck(cudaStreamSynchronize(p->st));
  }
  if (!p->sig_layer.empty() && !p->sig) p->sig = upload(p, sn);
  if (!p->zb) p->zb = upload(p, p->z_begin);

  const long long vol = (long long)p->nx * p->ny * nz;
  if (!p->Pb) {
    p->Pb = dalloc<double2>(p, vol);
    p->Qb = dalloc<double2>(p, vol);
    if (p->need_global) {
      p->Pg = dalloc<double2>(p, vol);
      p->Qg = dalloc<double2>(p, vol);
    }
  }
  const unsigned long long inf_bits = 0x7ff0000000000000ULL;
  ck(cudaMemcpyAsync(p->minpiv, &inf_bits, sizeof(inf_bits), cudaMemcpyHostToDevice, p->st));
  ck(cudaMemsetAsync(p->status, 0, sizeof(int), p->st));
  hz::zfactor(p->Pb, p->Qb, p->dx.lam_b, p->dy.lam_b, p->dx.skip, p->dy.skip, p->tzd, p->szs, p->coff,
              p->mz, p->nx, p->ny, nz, p->minpiv, p->status, p->st);
  if (p->need_global)
    hz::zfactor(p->Pg, p->Qg, p->dx.lam_g, p->dy.lam_g, nullptr, nullptr, p->tzd, p->szs, p->coff,
                nullptr, p->nx, p->ny, nz, p->minpiv, p->status, p->st);
  ck(cudaGetLastError());
  int status = 0;
  unsigned long long mp = 0;
  ck(cudaMemcpyAsync(&status, p->status, sizeof(int), cudaMemcpyDeviceToHost, p->st));
  ck(cudaMemcpyAsync(&mp, p->minpiv, sizeof(mp), cudaMemcpyDeviceToHost, p->st));
  ck(cudaStreamSynchronize(p->st));
  double mpd;
  std::memcpy(&mpd, &mp, sizeof(mpd));
  p->info.min_abs_pivot = mpd;
  if (status) throw Fail{(hz_status)status};
}

// Element counts of the workspace buffers of a solve of R right-hand sides: 17 double2
// buffers in the order FT, G, V, cX, vX, cY, vY, rX, rY, aX, bY, cg, dg, wX, wY, alX, alY,
// then the partial-sum doubles and the volume (for RHO).
struct WsSizes {
  long long c[17];
  long long partial;
  long long vol;
};
WsSizes ws_sizes(hz_plan_t p, int R) {
  WsSizes z{};
  const long long vol = (long long)p->nx * p->ny * p->nz * R;
  const long long zr = (long long)p->nz * R;
  const long long nIx = (long long)p->ax.iface.size(), nIy = (long long)p->ay.iface.size();
  const long long X = zr * nIx * p->ny, Y = zr * nIy * p->nx;
  const long long v[17] = {vol, vol, vol, 2 * X, 2 * X, 2 * Y, 2 * Y, X, Y, X, Y, X, Y, X, Y, X, Y};
  for (int i = 0; i < 17; ++i) z.c[i] = std::max(v[i], 1LL);
  hz::StencilArgs sa;
  sa.nx = p->nx; sa.ny = p->ny; sa.nz = p->nz; sa.nrhs = R;
  z.partial = 2LL * R * hz::stencil_parts(sa) + 2;
  z.vol = vol;
  return z;
}

double2** ws_slots(Workspace& w, int i) {
  double2** s[17] = {&w.FT, &w.G, &w.V, &w.cX, &w.vX, &w.cY, &w.vY, &w.rX, &w.rY, &w.aX, &w.bY,
                     &w.cg, &w.dg, &w.wX, &w.wY, &w.alX, &w.alY};
  return s[i];
}

void ensure_ws(hz_plan_t p, int R) {
  Workspace& w = p->ws;
  if (w.cap >= R) return;
  double2** bufs[] = {&w.FT, &w.G, &w.V, &w.cX, &w.vX, &w.cY, &w.vY, &w.rX, &w.rY, &w.aX, &w.bY,
                      &w.cg, &w.dg, &w.wX, &w.wY, &w.alX, &w.alY};
  for (double2** b : bufs) { dfree(p, *b); *b = nullptr; }
  dfree(p, w.partial); dfree(p, w.norms);
  const long long vol = (long long)p->nx * p->ny * p->nz * R;
  const long long zr = (long long)p->nz * R;
  const int nIx = (int)p->ax.iface.size(), nIy = (int)p->ay.iface.size();
  w.FT = dalloc<double2>(p, vol);
  w.G = dalloc<double2>(p, vol);
  w.V = dalloc<double2>(p, vol);
  w.cX = dalloc<double2>(p, zr * 2 * nIx * p->ny);
  w.vX = dalloc<double2>(p, zr * 2 * nIx * p->ny);
  w.cY = dalloc<double2>(p, zr * 2 * nIy * p->nx);
  w.vY = dalloc<double2>(p, zr * 2 * nIy * p->nx);
  w.rX = dalloc<double2>(p, zr * nIx * p->ny);
  w.rY = dalloc<double2>(p, zr * nIy * p->nx);
  w.aX = dalloc<double2>(p, zr * nIx * p->ny);
  w.bY = dalloc<double2>(p, zr * nIy * p->nx);
  w.cg = dalloc<double2>(p, zr * nIx * p->ny);
  w.dg = dalloc<double2>(p, zr * nIy * p->nx);
  w.wX = dalloc<double2>(p, zr * nIx * p->ny);
  w.wY = dalloc<double2>(p, zr * nIy * p->nx);
  w.alX = dalloc<double2>(p, zr * nIx * p->ny);
  w.alY = dalloc<double2>(p, zr * nIy * p->nx);
  {
    hz::StencilArgs sa;
    sa.nx = p->nx; sa.ny = p->ny; sa.nz = p->nz; sa.nrhs = R;
    w.partial = dalloc<double>(p, (size_t)2 * R * hz::stencil_parts(sa) + 2);
  }
  w.norms = dalloc<double>(p, (size_t)4 * R);                 // two sets of residual sums
  w.cap = R;
  if (w.rho_cap) { dfree(p, w.RHO); w.RHO = nullptr; w.rho_cap = 0; }
  if (w.f2_cap) { dfree(p, w.F2); w.F2 = nullptr; w.f2_cap = 0; }
  if (w.hu_cap) { dfree(p, w.HU); w.HU = nullptr; w.hu_cap = 0; }
}

double2* ensure_extra(hz_plan_t p, double2*& buf, int& cap, int R) {
  if (cap < R) {
    dfree(p, buf);
    buf = dalloc<double2>(p, (long long)p->nx * p->ny * p->nz * R);
    cap = R;
  }
  return buf;
}

hz::IfaceArgs iface_args(hz_plan_t p, int R) {
  hz::IfaceArgs a;
  a.nx = p->nx; a.ny = p->ny; a.nz = p->nz; a.nrhs = R;
  a.nIx = (int)p->ax.iface.size(); a.nIy = (int)p->ay.iface.size();
  a.xif = p->dx.ifc; a.yif = p->dy.ifc;
  a.isx = p->dx.skip; a.isy = p->dy.skip;
  a.mx = p->dx.m; a.my = p->dy.m; a.mz = p->mz;
  a.ihx = p->dx.ih; a.ihy = p->dy.ih;
  a.sig = p->sig;
  return a;
}

// The x-side and y-side interface chains are independent: the y side runs on the
// plan's second stream between fork() and join().
void fork(hz_plan_t p, cudaStream_t st) {
  ck(cudaEventRecord(p->ev_fork, st));
  ck(cudaStreamWaitEvent(p->side, p->ev_fork, 0));
}
void join(hz_plan_t p, cudaStream_t st) {
  ck(cudaEventRecord(p->ev_join, p->side));
  ck(cudaStreamWaitEvent(st, p->ev_join, 0));
}

// One pass of steps 1-7: u (=|+=) S(f).  lo = FP32 bulk transforms (mixed path).
void solve_core(hz_plan_t p, Workspace& w, cudaStream_t st, const double2* f, double2* u, int R, bool lo,
                int store, int conj_out) {
  const int nx = p->nx, ny = p->ny, nz = p->nz;
  const long long planes = (long long)R * nz;
  const int nIx = (int)p->ax.iface.size(), nIy = (int)p->ay.iface.size();
  // Mixed path with tensor-core transforms: the mode-space volumes (the transformed right-hand
  // side f~, the half-transformed planes in G and the z-sweep results) are complex64, since
  // the transforms that produce them accumulate in FP32 and the ones that consume them split
  // FP32 values into TF32 parts; the z eliminations keep FP64 forward values in V's buffer.
  // FT's buffer holds f~ (first half) and the z-sweep results (second half).
  const bool c64 = lo && p->use_tc && !conj_out;
  float2* const FT32 = reinterpret_cast<float2*>(w.FT);
  float2* const V32 = FT32 + planes * nx * ny;
  float2* const G32 = reinterpret_cast<float2*>(w.G);
  // bulk transforms: FP64 DFMA, or (mixed path) 3xTF32 on the tensor cores
  auto bulk = [&](const hz::XformSet& xs, const hz::TCSet& ts, const void* in, int in32, void* out, int out32,
                  int rpp, int trans, int store_mode, int conj, const signed char* skip) {
    if (in32 || out32 || (lo && p->use_tc && !conj)) {
      // uniform blocks by the FP32 fast sine transform, the others on the tensor cores
      const bool fs = p->fast_sine32 && xs.dst.nblk > 0 && (in32 || out32);
      if (fs && !hz::dst_f32(xs.dst, in, in32, out, out32, rpp, planes, xs.ncols, trans, store_mode, skip, st))
        throw Fail{HZ_ERR_ARG};
      if (!hz::xform_tc(ts, in, in32, out, out32, rpp, planes, trans, store_mode, skip, p->status, st,
                        p->opts.precision == HZ_MIXED_TF32 ? 1 : 3, fs, p->tc_real))
        throw Fail{HZ_ERR_ARG};
    } else if (!lo) {
      hz::xform_f64(xs, static_cast<const double2*>(in), static_cast<double2*>(out), rpp, planes, trans,
                    store_mode, conj, skip, st, p->fast_sine, p->xf_tile);
    } else {
      hz::xform_f32(xs, static_cast<const double2*>(in), static_cast<double2*>(out), rpp, planes, trans,
                    store_mode, conj, skip, st, p->xf_tile);
    }
  };
  // The interface-row transforms below are non-transposed, so their rows are
  // flattened across planes (one launch row tile covers 32 rows of any planes).
  // On the mixed path the interface transforms of steps 3, 5 and 6 (contractions with
  // eigenvector rows, short row transforms, the rank-|I| right-hand sides) run in FP32
  // like the bulk transforms; the z eliminations, the interface residual and the
  // refinement residual stay FP64.
  auto rowx = [&](const hz::XformSet& xs, const double2* in, double2* out, long long rows, cudaStream_t s) {
    if (lo) hz::xform_f32(xs, in, out, (int)rows, 1, 0, hz::XS_STORE, 0, nullptr, s, p->xf_tile);
    else hz::xform_f64(xs, in, out, (int)rows, 1, 0, hz::XS_STORE, 0, nullptr, s, p->fast_sine, p->xf_tile);
  };
  // contractions of the current z-sweep result (complex64 in V32, or complex128 in V)
  auto crows = [&](const AxisDev& d, double2* out, bool edge, int nslots, cudaStream_t s) {
    const int2* rng = edge ? d.edge_rng : d.grng;
    if (c64) {
      if (!edge && hz::contract_all(true, V32, out, d.gcoef32, nx, ny, nslots, planes, s)) return;
      hz::contract_rows(V32, out, edge ? d.edge_coef32 : d.gcoef32, rng, nx, ny, nslots, planes, s);
      return;
    }
    // FP32: one pass over V for all slots; FP64 stays per slot (bound by the FP64 pipe, where
    // one pass saves no work but gives fewer threads)
    if (!edge && lo && hz::contract_all(true, w.V, out, d.gcoef32, nx, ny, nslots, planes, s)) return;
    if (lo) hz::contract_rows(w.V, out, edge ? d.edge_coef32 : d.gcoef32, rng, nx, ny, nslots, planes, s);
    else hz::contract_rows(w.V, out, edge ? d.edge_coef : d.gcoef, rng, nx, ny, nslots, planes, s,
                           edge ? d.edge_real : d.g_real);
  };
  auto ccols = [&](const AxisDev& d, double2* out, bool edge, int nslots, cudaStream_t s) {
    const int2* rng = edge ? d.edge_rng : d.grng;
    if (c64) {
      if (!edge && hz::contract_all(false, V32, out, d.gcoef32, nx, ny, nslots, planes, s)) return;
      hz::contract_cols(V32, out, edge ? d.edge_coef32 : d.gcoef32, rng, nx, ny, nslots, planes, s);
      return;
    }
    if (!edge && lo && hz::contract_all(false, w.V, out, d.gcoef32, nx, ny, nslots, planes, s)) return;
    if (lo) hz::contract_cols(w.V, out, edge ? d.edge_coef32 : d.gcoef32, rng, nx, ny, nslots, planes, s);
    else hz::contract_cols(w.V, out, edge ? d.edge_coef : d.gcoef, rng, nx, ny, nslots, planes, s,
                           edge ? d.edge_real : d.g_real);
  };
  // Step 1: f~ = (W_x^T M_x) (x) (W_y^T M_y) f per plane; rows j -> G[i][j] -> FT[i][j]
  {
    Stage t(p, st, HZ_STAGE_FWD);
    if (c64) {
      bulk(p->dx.fwd, p->dx.tfwd, f, 0, G32, 1, ny, 1, hz::XS_STORE, 0, p->dy.skip);
      bulk(p->dy.fwd, p->dy.tfwd, G32, 1, FT32, 1, nx, 0, hz::XS_STORE, 0, p->dx.skip);
    } else {
      bulk(p->dx.fwd, p->dx.tfwd, f, 0, w.G, 0, ny, 1, hz::XS_STORE, 0, p->dy.skip);
      bulk(p->dy.fwd, p->dy.tfwd, w.G, 0, w.FT, 0, nx, 0, hz::XS_STORE, 0, p->dx.skip);
    }
  }

  hz::ZSolveArgs za;
  za.nx = nx; za.ny = ny; za.nz = nz; za.nrhs = R;
  za.real_cm = p->real_cm;
  za.skip_i = p->dx.skip; za.skip_j = p->dy.skip;
  za.rhs = w.FT; za.out = w.V;
  za.P = p->Pb; za.Q = p->Qb; za.cm = p->cm_b;
  za.rhs_per_thread = p->zs_rb;
  za.sms = p->sms;
  if (c64) { za.rhs32 = FT32; za.out32 = V32; za.scratch = w.V; }
  // Step 2: mode-wise z solves of every block (pass A)
  {
    Stage t(p, st, HZ_STAGE_PASS_A);
    hz::zsolve(za, st);
  }

  if (nIx + nIy > 0) {
    // Step 3: v at the nodes next to the interfaces
    std::unique_ptr<Stage> t3(new Stage(p, st, HZ_STAGE_EDGES));
    const cudaStream_t sy = p->side;
    fork(p, st);
    if (nIx) {
      crows(p->dx, w.cX, true, 2 * nIx, st);
      rowx(p->dy.inv, w.cX, w.vX, 2 * nIx * planes, st);
    }
    if (nIy) {
      ccols(p->dy, w.cY, true, 2 * nIy, sy);
      rowx(p->dx.inv, w.cY, w.vY, 2 * nIy * planes, sy);
    }
    join(p, st);
    t3.reset();
    // Step 4: r = M f - A v on the interfaces
    hz::IfaceArgs ia = iface_args(p, R);
    {
      Stage t(p, st, HZ_STAGE_IRES);
      hz::iface_residual(ia, f, w.vX, w.vY, w.rX, w.rY, st);
    }
    // Step 5: w on the interfaces through the whole-axis eigenbasis
    std::unique_ptr<Stage> t5(new Stage(p, st, HZ_STAGE_GLOBAL));
    fork(p, st);
    if (nIx) rowx(p->dy.gfwd, w.rX, w.aX, nIx * planes, st);
    if (nIy) rowx(p->dx.gfwd, w.rY, w.bY, nIy * planes, sy);
    join(p, st);
    hz::GlobalRhsArgs ga;
    ga.nx = nx; ga.ny = ny; ga.nz = nz; ga.nrhs = R; ga.nIx = nIx; ga.nIy = nIy;
    ga.aX = w.aX; ga.bY = w.bY; ga.WgxI = p->dx.gcoef; ga.WgyI = p->dy.gcoef;
    ga.real_x = p->dx.g_real ? 1 : 0; ga.real_y = p->dy.g_real ? 1 : 0;
    if (lo) { ga.WgxI32 = p->dx.gcoef32; ga.WgyI32 = p->dy.gcoef32; }
    hz::ZSolveArgs zg = za;
    zg.skip_i = nullptr; zg.skip_j = nullptr;
    zg.rhs = w.G; zg.out = w.V;                     // w~ (v~ in V is no longer needed)
    zg.P = p->Pg; zg.Q = p->Qg; zg.cm = p->cm_g;
    if (c64) zg.rhs32 = G32;
    if (c64) {
      // complex64 copies of the interface transforms (cg, dg are free until the contractions)
      float2* aX32 = reinterpret_cast<float2*>(w.cg);
      float2* bY32 = reinterpret_cast<float2*>(w.dg);
      hz::to_c64_copy(w.aX, aX32, (long long)nIx * ny * planes, st);
      hz::to_c64_copy(w.bY, bY32, (long long)nIy * nx * planes, st);
      // r~ formed inside the sweep where the sweep can (FP32, from the complex64 interface
      // transforms), else by global_rhs into G
      zg.gen.kind = 1;
      zg.gen.nIx = nIx; zg.gen.nIy = nIy;
      zg.gen.aX32 = aX32; zg.gen.bY32 = bY32;
      zg.gen.wx32 = p->dx.gcoef32; zg.gen.wy32 = p->dy.gcoef32;
      if (!hz::zsolve_forms_rhs(zg)) {
        zg.gen.kind = 0;
        ga.aX32 = aX32;
        ga.bY32 = bY32;
        hz::global_rhs(ga, G32, st);
      }
    } else {
      hz::global_rhs(ga, w.G, st);
    }
    hz::zsolve(zg, st);
    fork(p, st);
    if (nIx) {
      crows(p->dx, w.cg, false, nIx, st);
      rowx(p->dy.ginv, w.cg, w.wX, nIx * planes, st);
      // Step 6 (x interfaces): forward y-transform of w on the interface rows
      rowx(p->dy.fwd, w.wX, w.alX, nIx * planes, st);
    }
    if (nIy) {
      ccols(p->dy, w.dg, false, nIy, sy);
      rowx(p->dx.ginv, w.dg, w.wY, nIy * planes, sy);
      rowx(p->dx.fwd, w.wY, w.alY, nIy * planes, sy);
    }
    join(p, st);
    t5.reset();
    // Step 6: pass B, (Tz + s S_z) u~ = M_z f~ + g~ with g~ formed from the interface data
    Stage t6(p, st, HZ_STAGE_PASS_B);
    hz::BoundaryArgs ba;
    ba.nx = nx; ba.ny = ny; ba.nz = nz; ba.nrhs = R; ba.nIx = nIx; ba.nIy = nIy;
    ba.skip_i = p->dx.skip; ba.skip_j = p->dy.skip; ba.sig = p->sig;
    ba.alphaX = w.alX; ba.alphaY = w.alY;
    ba.gxl = p->dx.gl; ba.gxr = p->dx.gr; ba.gyl = p->dy.gl; ba.gyr = p->dy.gr;
    ba.cxl = p->dx.cl; ba.cxr = p->dx.cr; ba.cyl = p->dy.cl; ba.cyr = p->dy.cr;
    ba.real_x = p->dx.lr_real ? 1 : 0; ba.real_y = p->dy.lr_real ? 1 : 0;
    if (lo) { ba.cxl32 = p->dx.cl32; ba.cxr32 = p->dx.cr32; ba.cyl32 = p->dy.cl32; ba.cyr32 = p->dy.cr32; }
    if (c64) {
      // complex64 copies of the boundary data (aX, bY are free after step 5); f~ + g~ in FP32
      float2* alX32 = reinterpret_cast<float2*>(w.aX);
      float2* alY32 = reinterpret_cast<float2*>(w.bY);
      hz::to_c64_copy(w.alX, alX32, (long long)nIx * ny * planes, st);
      hz::to_c64_copy(w.alY, alY32, (long long)nIy * nx * planes, st);
      // f~ + g~ / M_z formed inside the sweep where the sweep can (FP32; f~ itself is left as
      // it is), else by boundary_rhs into f~
      hz::ZSolveArgs zb = za;
      zb.gen.kind = 2;
      zb.gen.nIx = nIx; zb.gen.nIy = nIy;
      zb.gen.aX32 = alX32; zb.gen.bY32 = alY32;
      zb.gen.gxl = p->dx.gl; zb.gen.gxr = p->dx.gr; zb.gen.gyl = p->dy.gl; zb.gen.gyr = p->dy.gr;
      zb.gen.cxl32 = p->dx.cl32; zb.gen.cxr32 = p->dx.cr32; zb.gen.cyl32 = p->dy.cl32; zb.gen.cyr32 = p->dy.cr32;
      zb.gen.sig = p->sig;
      if (!hz::zsolve_forms_rhs(zb)) {
        zb.gen.kind = 0;
        ba.alphaX32 = alX32;
        ba.alphaY32 = alY32;
        hz::boundary_rhs(ba, FT32, st);             // f~ + g~ / M_z, in place
      }
      hz::zsolve(zb, st);
    } else {
      hz::boundary_rhs(ba, w.FT, st);
      hz::zsolve(za, st);
    }
  }
  // Step 7: u = W_x (x) W_y u~ in the blocks; u = w on the interfaces
  {
    Stage t(p, st, HZ_STAGE_INV);
    if (c64) {
      bulk(p->dy.inv, p->dy.tinv, V32, 1, G32, 1, nx, 1, hz::XS_STORE, 0, p->dx.skip);
      bulk(p->dx.inv, p->dx.tinv, G32, 1, u, 0, ny, 0, store, conj_out, p->dy.skip);
    } else {
      bulk(p->dy.inv, p->dy.tinv, w.V, 0, w.G, 0, nx, 1, hz::XS_STORE, 0, p->dx.skip);
      bulk(p->dx.inv, p->dx.tinv, w.G, 0, u, 0, ny, 0, store, conj_out, p->dy.skip);
    }
  }
  if (nIx + nIy > 0) {
    Stage t(p, st, HZ_STAGE_IFACE_OUT);
    hz::IfaceArgs ia = iface_args(p, R);
    hz::write_iface(ia, w.wX, w.wY, u, conj_out, store == hz::XS_ACCUM, st);
  }
  ck(cudaGetLastError());
}

hz::StencilArgs stencil_args(hz_plan_t p, int R) {
  hz::StencilArgs a;
  a.nx = p->nx; a.ny = p->ny; a.nz = p->nz; a.nrhs = R;
  a.kxs = p->dx.ks; a.kys = p->dy.ks; a.tzs = p->tzs; a.sig = p->sig;
  a.mx = p->dx.m; a.my = p->dy.m; a.mz = p->mz;
  a.cxy = p->cxy; a.w2xy = p->w2xy; a.w2z = p->w2z;
  a.rx = p->dx.kreal; a.ry = p->dy.kreal; a.rz = p->rz;
  return a;
}

// Enqueue rho = f - M^{-1} A u (rho may be NULL) and the per-RHS sums (|M rho|^2, |M f|^2)
// into norms[2R] (no synchronisation: usable inside a stream capture).
void residual_enqueue(hz_plan_t p, Workspace& w, cudaStream_t st, const double2* f, const double2* u,
                      double2* rho, double* norms, int R, int fnorm) {
  hz::StencilArgs a = stencil_args(p, R);
  const int parts = hz::stencil_parts(a);
  Stage t(p, st, HZ_STAGE_RESID);
  hz::stencil_residual(a, f, u, rho, w.partial, fnorm, st);
  hz::finish_norms(w.partial, parts, R, norms, st);
}

// Relative residuals from the sums of residual_enqueue; fnorm2 caches ||M f||^2.
double residual_from_sums(const std::vector<double>& nrm, int R, std::vector<double>* per_rhs,
                          std::vector<double>& fnorm2) {
  if (fnorm2.empty()) {
    fnorm2.resize(R);
    for (int r = 0; r < R; ++r) fnorm2[r] = nrm[2 * r + 1];
  }
  double worst = 0.0;
  if (per_rhs) per_rhs->assign(R, 0.0);
  for (int r = 0; r < R; ++r) {
    const double rel = fnorm2[r] > 0 ? std::sqrt(nrm[2 * r] / fnorm2[r]) : std::sqrt(nrm[2 * r]);
    if (!std::isfinite(rel)) throw Fail{HZ_ERR_NONFINITE};
    if (per_rhs) (*per_rhs)[r] = rel;
    worst = std::max(worst, rel);
  }
  return worst;
}

// rho = f - M^{-1} A u (rho may be NULL); returns max over RHS of ||M rho|| / ||M f||.
// fnorm2 caches ||M f||^2 per RHS across calls with the same f (computed when empty).
double residual_core(hz_plan_t p, const double2* f, const double2* u, double2* rho, int R,
                     std::vector<double>* per_rhs, std::vector<double>& fnorm2) {
  residual_enqueue(p, p->ws, p->st, f, u, rho, p->ws.norms, R, fnorm2.empty() ? 1 : 0);
  ck(cudaGetLastError());
  std::vector<double> nrm(2 * R);
  ck(cudaMemcpyAsync(nrm.data(), p->ws.norms, 2 * R * sizeof(double), cudaMemcpyDeviceToHost, p->st));
  ck(cudaStreamSynchronize(p->st));
  return residual_from_sums(nrm, R, per_rhs, fnorm2);
}

// Full solve: FP64 single pass, or mixed with FP64 refinement.
void solve_full_impl(hz_plan_t p, const double2* f, double2* u, int R, int conj_out);

void solve_full(hz_plan_t p, const double2* f, double2* u, int R, int conj_out) {
  const long long l0 = hz::launch_count();
  solve_full_impl(p, f, u, R, conj_out);
  p->info.kernel_launches += hz::launch_count() - l0;
  if (p->timing) collect_stages(p);
}

void solve_full_impl(hz_plan_t p, const double2* f, double2* u, int R, int conj_out) {
  ensure_ws(p, R);
  p->info.refinements = 0;
  p->info.rel_residual = -1.0;
  if (p->opts.precision == HZ_FP64) {
    solve_core(p, p->ws, p->st, f, u, R, false, hz::XS_STORE, conj_out);
    ck(cudaStreamSynchronize(p->st));
    return;
  }
  const double2* fin = f;
  if (f == u) {   // refinement needs f after u is written
    double2* f2 = ensure_extra(p, p->ws.F2, p->ws.f2_cap, R);
    ck(cudaMemcpyAsync(f2, f, sizeof(double2) * (size_t)p->nx * p->ny * p->nz * R,
                       cudaMemcpyDeviceToDevice, p->st));
    fin = f2;
  }
  double2* rho = ensure_extra(p, p->ws.RHO, p->ws.rho_cap, R);
  ck(cudaMemsetAsync(p->status, 0, sizeof(int), p->st));
  solve_core(p, p->ws, p->st, fin, u, R, true, hz::XS_STORE, 0);
  std::vector<double> fn2;
  double rel;
  int it = 0;
  if (p->opts.max_refine >= 1) {
    // The FP32 transforms leave a residual far above any useful rtol, so the first correction
    // is enqueued behind the first residual without waiting for it; both norms come back
    // with one synchronisation.
    double* n1 = p->ws.norms;
    double* n2 = p->ws.norms + 2 * R;
    residual_enqueue(p, p->ws, p->st, fin, u, rho, n1, R, 1);
    solve_core(p, p->ws, p->st, rho, u, R, true, hz::XS_ACCUM, 0);
    residual_enqueue(p, p->ws, p->st, fin, u, rho, n2, R, 0);
    ck(cudaGetLastError());
    std::vector<double> nrm(4 * R);
    ck(cudaMemcpyAsync(nrm.data(), n1, 4 * R * sizeof(double), cudaMemcpyDeviceToHost, p->st));
    ck(cudaStreamSynchronize(p->st));
    residual_from_sums(std::vector<double>(nrm.begin(), nrm.begin() + 2 * R), R, nullptr, fn2);
    rel = residual_from_sums(std::vector<double>(nrm.begin() + 2 * R, nrm.end()), R, nullptr, fn2);
    it = 1;
  } else {
    rel = residual_core(p, fin, u, rho, R, nullptr, fn2);
  }
  while (rel > p->opts.rtol && it < p->opts.max_refine) {
    solve_core(p, p->ws, p->st, rho, u, R, true, hz::XS_ACCUM, 0);
    rel = residual_core(p, fin, u, rho, R, nullptr, fn2);
    ++it;
  }
  p->info.refinements = it;
  p->info.rel_residual = rel;
  int status = 0;
  ck(cudaMemcpyAsync(&status, p->status, sizeof(int), cudaMemcpyDeviceToHost, p->st));
  ck(cudaStreamSynchronize(p->st));
  if (status) throw Fail{(hz_status)status};
  if (conj_out) {
    hz::conj_inplace(u, (long long)p->nx * p->ny * p->nz * R, p->st);
    ck(cudaStreamSynchronize(p->st));
  }
  if (rel > p->opts.rtol) throw Fail{HZ_ERR_NOT_CONVERGED};
}

void release(hz_plan_t p) {
  for (void* a : p->allocs) cudaFree(a);
  p->allocs.clear();
  for (cudaEvent_t e : p->ev_pool) cudaEventDestroy(e);
  p->ev_pool.clear();
  if (p->side) cudaStreamDestroy(p->side);
  if (p->ev_fork) cudaEventDestroy(p->ev_fork);
  if (p->ev_join) cudaEventDestroy(p->ev_join);
  if (p->cst) cudaStreamDestroy(p->cst);
  if (p->cst2) cudaStreamDestroy(p->cst2);
  for (cudaEvent_t& e : p->ev_in) {
    if (e) cudaEventDestroy(e);
    e = nullptr;
  }
  p->side = nullptr;
  p->ev_fork = p->ev_join = nullptr;
  p->cst = p->cst2 = nullptr;
}

}  // namespace

// ---------------------------------------------------------------------------
// Batches: many (plan, nrhs) solves replayed as one CUDA graph
// ---------------------------------------------------------------------------
namespace {

// Time the plan's kernel variants (z-sweep variant 1, 2 or 3; on the mixed path tensor-core or
// CUDA-core bulk transforms and the real-table or interleaved tensor-core kernel; with uniform
// blocks the fast sine transform or the dense product; 16 or 64 data rows per CTA of the dense
// CUDA-core transforms) with three solves each on workspace w and stream st, keep the fastest;
// returns z_sweep + 10 tc + 100 fast_sine + 1000 real_tables + 10000 tile (1: 16 rows, 2: 64)
// of the choice.  f and out are device buffers of nrhs RHS.
int tune_plan(hz_plan_t p, Workspace& w, cudaStream_t st, const double2* f, double2* out, int nrhs) {
  const bool mixed = p->opts.precision != HZ_FP64;
  const bool timing = p->timing;
  p->timing = false;
  cudaEvent_t e0, e1;
  ck(cudaEventCreate(&e0));
  ck(cudaEventCreate(&e1));
  float best = 1e30f;
  int best_rb = p->zs_rb;
  int best_tile = p->xf_tile;
  bool best_tc = p->use_tc;
  bool& fsref = mixed ? p->fast_sine32 : p->fast_sine;     // the fast-sine choice of this path
  bool best_fs = fsref;
  bool best_tr = p->tc_real;
  const int tr_lo = (mixed && p->has_real_tc) ? 0 : (p->tc_real ? 1 : 0);
  const int tr_hi = (mixed && p->has_real_tc) ? 1 : tr_lo;
  const int fs_lo = p->has_dst ? 0 : (fsref ? 1 : 0);
  const int fs_hi = p->has_dst ? 1 : fs_lo;
  for (int tile : {64, 16})
  for (int tr = tr_lo; tr <= tr_hi; ++tr)
  for (int fs = fs_lo; fs <= fs_hi; ++fs)
  for (int rb = 1; rb <= 3; ++rb)
    for (int tc = (mixed || !p->tc_ok) ? 0 : 1; tc <= (p->tc_ok ? 1 : 0); ++tc) {
      p->xf_tile = tile;
      p->tc_real = tr != 0;
      fsref = fs != 0;
      p->zs_rb = rb;
      p->use_tc = tc != 0;
      solve_core(p, w, st, f, out, nrhs, mixed, hz::XS_STORE, 0);   // warm-up
      ck(cudaEventRecord(e0, st));
      for (int rep = 0; rep < 3; ++rep) solve_core(p, w, st, f, out, nrhs, mixed, hz::XS_STORE, 0);
      ck(cudaEventRecord(e1, st));
      ck(cudaEventSynchronize(e1));
      float ms = 0.f;
      ck(cudaEventElapsedTime(&ms, e0, e1));
      if (ms < best) { best = ms; best_rb = rb; best_tc = tc != 0; best_fs = fs != 0; best_tr = tr != 0; best_tile = tile; }
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  p->zs_rb = best_rb;
  p->xf_tile = best_tile;
  p->use_tc = best_tc;
  fsref = best_fs;
  p->tc_real = best_tr;
  p->timing = timing;
  return best_rb + (best_tc ? 10 : 0) + (best_fs ? 100 : 0) + (best_tr ? 1000 : 0) + (best_tile == 16 ? 10000 : 20000);
}

}  // namespace

struct hz_batch_s {
  std::vector<hz_plan_t> plans;
  std::vector<int> nrhs;
  std::vector<int> lane_of;                 // item -> lane
  int nlanes = 1;
  cudaStream_t s0 = nullptr;
  std::vector<cudaStream_t> lanes;
  std::vector<Workspace> ws;                // one per lane, sized for its largest item
  std::vector<double2*> rho;                // one per lane
  double* norms = nullptr;                  // [item][4 R]: first and final residual sums
  std::vector<long long> norm_off;
  std::vector<void*> allocs;
  cudaEvent_t fork = nullptr;
  std::vector<cudaEvent_t> joins;
  cudaGraphExec_t exec = nullptr;
  std::vector<const void*> graph_f, graph_u;   // pointers the graph was captured with
  double last_ms = 0.0;
  long long launches_per_replay = 0;
};

namespace {

void bfree(hz_batch_t b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  b->exec = nullptr;
  for (void* a : b->allocs) cudaFree(a);
  b->allocs.clear();
  for (cudaStream_t s : b->lanes) cudaStreamDestroy(s);
  b->lanes.clear();
  if (b->fork) cudaEventDestroy(b->fork);
  b->fork = nullptr;
  for (cudaEvent_t e : b->joins) cudaEventDestroy(e);
  b->joins.clear();
}

template <typename T>
T* balloc(hz_batch_t b, long long count) {
  void* ptr = nullptr;
  ck(cudaMalloc(&ptr, (size_t)std::max(count, 1LL) * sizeof(T)));
  b->allocs.push_back(ptr);
  return static_cast<T*>(ptr);
}

// Lane workspaces (each sized for the largest item of its lane), streams and events.
void batch_setup(hz_batch_t b, int nlanes) {
  bfree(b);
  const int n = (int)b->plans.size();
  b->nlanes = std::max(1, std::min(nlanes, n));
  // greedy balance of estimated work (unknowns x RHS) over the lanes
  std::vector<int> order(n);
  for (int i = 0; i < n; ++i) order[i] = i;
  auto cost = [&](int i) { return (double)b->plans[i]->nx * b->plans[i]->ny * b->plans[i]->nz * b->nrhs[i]; };
  std::sort(order.begin(), order.end(), [&](int a, int c) { return cost(a) > cost(c); });
  std::vector<double> load(b->nlanes, 0.0);
  b->lane_of.assign(n, 0);
  for (int i : order) {
    const int l = (int)(std::min_element(load.begin(), load.end()) - load.begin());
    b->lane_of[i] = l;
    load[l] += cost(i);
  }
  b->ws.assign(b->nlanes, Workspace{});
  b->rho.assign(b->nlanes, nullptr);
  for (int l = 0; l < b->nlanes; ++l) {
    WsSizes mx{};
    for (int i = 0; i < n; ++i) {
      if (b->lane_of[i] != l) continue;
      const WsSizes z = ws_sizes(b->plans[i], b->nrhs[i]);
      for (int q = 0; q < 17; ++q) mx.c[q] = std::max(mx.c[q], z.c[q]);
      mx.partial = std::max(mx.partial, z.partial);
      mx.vol = std::max(mx.vol, z.vol);
    }
    for (int q = 0; q < 17; ++q) *ws_slots(b->ws[l], q) = balloc<double2>(b, mx.c[q]);
    b->ws[l].partial = balloc<double>(b, mx.partial);
    b->rho[l] = balloc<double2>(b, mx.vol);
  }
  b->norm_off.assign(n, 0);
  long long tot = 0;
  for (int i = 0; i < n; ++i) {
    b->norm_off[i] = tot;
    tot += 4LL * b->nrhs[i];
  }
  b->norms = balloc<double>(b, tot);
  ck(cudaStreamCreateWithFlags(&b->s0, cudaStreamNonBlocking));
  b->lanes.push_back(b->s0);   // lane 0 runs on the capture origin stream
  for (int l = 1; l < b->nlanes; ++l) {
    cudaStream_t s;
    ck(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    b->lanes.push_back(s);
  }
  ck(cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming));
  b->joins.resize(b->nlanes);
  for (auto& e : b->joins) ck(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
}

// Enqueue every item of the batch on its lane (inside a stream capture).
void batch_enqueue(hz_batch_t b, const hz_c128* const* f_dev, hz_c128* const* u_dev) {
  ck(cudaEventRecord(b->fork, b->s0));
  for (int l = 1; l < b->nlanes; ++l) ck(cudaStreamWaitEvent(b->lanes[l], b->fork, 0));
  for (int i = 0; i < (int)b->plans.size(); ++i) {
    hz_plan_t p = b->plans[i];
    const int l = b->lane_of[i], R = b->nrhs[i];
    cudaStream_t st = b->lanes[l];
    Workspace& w = b->ws[l];
    const double2* f = reinterpret_cast<const double2*>(f_dev[i]);
    double2* u = reinterpret_cast<double2*>(u_dev[i]);
    double* nrm = b->norms + b->norm_off[i];
    if (p->opts.precision != HZ_FP64) {
      // first solve, its residual (with ||M f||), one correction, the final residual
      solve_core(p, w, st, f, u, R, true, hz::XS_STORE, 0);
      residual_enqueue(p, w, st, f, u, b->rho[l], nrm, R, 1);
      solve_core(p, w, st, b->rho[l], u, R, true, hz::XS_ACCUM, 0);
      residual_enqueue(p, w, st, f, u, nullptr, nrm + 2 * R, R, 1);
    } else {
      solve_core(p, w, st, f, u, R, false, hz::XS_STORE, 0);
      residual_enqueue(p, w, st, f, u, nullptr, nrm + 2 * R, R, 1);
    }
  }
  for (int l = 1; l < b->nlanes; ++l) {
    ck(cudaEventRecord(b->joins[l], b->lanes[l]));
    ck(cudaStreamWaitEvent(b->s0, b->joins[l], 0));
  }
}

void batch_capture(hz_batch_t b, const hz_c128* const* f_dev, hz_c128* const* u_dev) {
  if (b->exec) {
    cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
  }
  for (hz_plan_t p : b->plans) p->timing = false;
  const long long l0 = hz::launch_count();
  ck(cudaStreamBeginCapture(b->s0, cudaStreamCaptureModeRelaxed));
  try {
    batch_enqueue(b, f_dev, u_dev);
  } catch (...) {
    cudaGraph_t g = nullptr;
    cudaStreamEndCapture(b->s0, &g);
    if (g) cudaGraphDestroy(g);
    throw;
  }
  cudaGraph_t g = nullptr;
  ck(cudaStreamEndCapture(b->s0, &g));
  const cudaError_t e = cudaGraphInstantiate(&b->exec, g, 0);
  cudaGraphDestroy(g);
  ck(e);
  b->launches_per_replay = hz::launch_count() - l0;
  const int n = (int)b->plans.size();
  b->graph_f.assign(f_dev, f_dev + n);
  b->graph_u.assign(u_dev, u_dev + n);
}

// Replay; returns per-item max relative residual (items that miss rtol are refined eagerly).
void batch_run(hz_batch_t b, const hz_c128* const* f_dev, hz_c128* const* u_dev, double* rel_host) {
  const int n = (int)b->plans.size();
  bool same = b->exec && (int)b->graph_f.size() == n;
  for (int i = 0; same && i < n; ++i) same = b->graph_f[i] == f_dev[i] && b->graph_u[i] == u_dev[i];
  if (!same) batch_capture(b, f_dev, u_dev);
  for (hz_plan_t p : b->plans) ck(cudaMemsetAsync(p->status, 0, sizeof(int), b->s0));
  cudaEvent_t e0, e1;
  ck(cudaEventCreate(&e0));
  ck(cudaEventCreate(&e1));
  ck(cudaEventRecord(e0, b->s0));
  ck(cudaGraphLaunch(b->exec, b->s0));
  ck(cudaEventRecord(e1, b->s0));
  ck(cudaStreamSynchronize(b->s0));
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  b->last_ms = ms;
  for (hz_plan_t p : b->plans) p->info.kernel_launches += 0;
  long long tot = b->norm_off.empty() ? 0 : b->norm_off.back() + 4LL * b->nrhs.back();
  std::vector<double> nrm(std::max(tot, 1LL));
  ck(cudaMemcpy(nrm.data(), b->norms, sizeof(double) * tot, cudaMemcpyDeviceToHost));
  for (int i = 0; i < n; ++i) {
    hz_plan_t p = b->plans[i];
    int status = 0;
    ck(cudaMemcpy(&status, p->status, sizeof(int), cudaMemcpyDeviceToHost));
    if (status) throw Fail{(hz_status)status};
    const int R = b->nrhs[i];
    std::vector<double> fn2(R), fin(2 * R);
    for (int r = 0; r < R; ++r) fn2[r] = nrm[b->norm_off[i] + 2 * r + 1];
    for (int q = 0; q < 2 * R; ++q) fin[q] = nrm[b->norm_off[i] + 2 * R + q];
    double rel = residual_from_sums(fin, R, nullptr, fn2);
    if (p->opts.precision != HZ_FP64 && rel > p->opts.rtol) {
      // finish on the plan's own stream and workspace: more corrections, eagerly
      const double2* f = reinterpret_cast<const double2*>(f_dev[i]);
      double2* u = reinterpret_cast<double2*>(u_dev[i]);
      ensure_ws(p, R);
      double2* rho = ensure_extra(p, p->ws.RHO, p->ws.rho_cap, R);
      int it = 0;
      rel = residual_core(p, f, u, rho, R, nullptr, fn2);
      while (rel > p->opts.rtol && it < p->opts.max_refine) {
        solve_core(p, p->ws, p->st, rho, u, R, true, hz::XS_ACCUM, 0);
        rel = residual_core(p, f, u, rho, R, nullptr, fn2);
        ++it;
      }
      if (rel > p->opts.rtol) throw Fail{HZ_ERR_NOT_CONVERGED};
    }
    if (rel_host) rel_host[i] = rel;
  }
}

}  // namespace

namespace hz {
// Read-only views of a plan for the allocation-free residual (hz_noalloc.cu).
StencilArgs plan_stencil_args(hz_plan_t p, int nrhs) { return stencil_args(p, nrhs); }
cudaStream_t plan_stream(hz_plan_t p) { return p->st; }
int plan_device(hz_plan_t p) { return p->device; }
}  // namespace hz

extern "C" {

const char* hz_status_str(hz_status s) {
  switch (s) {
    case HZ_OK: return "ok";
    case HZ_ERR_ARG: return "invalid argument";
    case HZ_ERR_EIG: return "eigen-decomposition failed its checks";
    case HZ_ERR_SINGULAR: return "zero or non-finite pivot in a z elimination";
    case HZ_ERR_NONFINITE: return "non-finite value";
    case HZ_ERR_NOT_CONVERGED: return "iterative refinement did not reach rtol";
    case HZ_ERR_OOM: return "device allocation failed";
    case HZ_ERR_CUDA: return "CUDA runtime error";
    case HZ_ERR_TIMEOUT: return "bounded device wait gave up";
  }
  return "unknown status";
}

hz_status hz_plan_create(const hz_grid* grid, const hz_layers* layers, const hz_blocks* blocks,
                         const hz_options* opts, hz_plan_t* out) {
  if (!out) return HZ_ERR_ARG;
  *out = nullptr;
  if (!grid || !layers || !grid->hx || !grid->hy || !grid->hz) return HZ_ERR_ARG;
  if (grid->nx < 1 || grid->ny < 1 || grid->nz < 1) return HZ_ERR_ARG;
  if (layers->nlayers < 1 || !layers->z_begin || !layers->k2) return HZ_ERR_ARG;
  const int nl = layers->nlayers;
  if (layers->z_begin[0] != 0 || layers->z_begin[nl] != grid->nz) return HZ_ERR_ARG;
  for (int L = 0; L < nl; ++L) {
    if (layers->z_begin[L + 1] <= layers->z_begin[L]) return HZ_ERR_ARG;
    if (!std::isfinite(layers->k2[L].re) || !std::isfinite(layers->k2[L].im)) return HZ_ERR_ARG;
    if (layers->sigma && !(layers->sigma[L] > 0.0 && std::isfinite(layers->sigma[L]))) return HZ_ERR_ARG;
  }
  if (opts && (opts->precision < HZ_FP64 || opts->precision > HZ_MIXED_TF32)) return HZ_ERR_ARG;
  const bool mixed = opts && opts->precision != HZ_FP64;
  int nbx = blocks ? blocks->nbx : 1, nby = blocks ? blocks->nby : 1;
  if (blocks && nbx == HZ_BLOCKS_AUTO) {
    if (blocks->x_iface) return HZ_ERR_ARG;
    nbx = auto_blocks(grid->nx, mixed);
  }
  if (blocks && nby == HZ_BLOCKS_AUTO) {
    if (blocks->y_iface) return HZ_ERR_ARG;
    nby = auto_blocks(grid->ny, mixed);
  }
  if (nbx < 1 || nby < 1 || nbx > grid->nx || nby > grid->ny) return HZ_ERR_ARG;
  if ((long long)grid->nx * grid->ny >= (1LL << 31)) return HZ_ERR_ARG;      // in-plane indices are 32-bit

  hz_plan_t p = new (std::nothrow) hz_plan_s();
  if (!p) return HZ_ERR_OOM;
  const auto t0 = std::chrono::steady_clock::now();
  p->nx = grid->nx; p->ny = grid->ny; p->nz = grid->nz; p->nlayers = nl;
  if (opts) p->opts = *opts;
  else { p->opts.precision = HZ_FP64; p->opts.rtol = 1e-8; p->opts.max_refine = 10; p->opts.cuda_stream = nullptr; }
  if (!(p->opts.rtol > 0)) p->opts.rtol = 1e-8;
  if (p->opts.max_refine < 0) p->opts.max_refine = 0;
  p->st = (cudaStream_t)p->opts.cuda_stream;
  p->hz.resize(grid->nz + 1);
  for (int k = 0; k <= grid->nz; ++k) {
    p->hz[k] = cd(grid->hz[k].re, grid->hz[k].im);
    if (!finite(p->hz[k]) || std::abs(p->hz[k]) == 0.0) { delete p; return HZ_ERR_ARG; }
  }
  p->z_begin.assign(layers->z_begin, layers->z_begin + nl + 1);
  p->k2base.resize(nl);
  for (int L = 0; L < nl; ++L) p->k2base[L] = cd(layers->k2[L].re, layers->k2[L].im);
  if (layers->sigma) p->sig_layer.assign(layers->sigma, layers->sigma + nl);

  p->info.nbx = nbx;
  p->info.nby = nby;
  hz_status s = build_axis(p->ax, grid->nx, grid->hx, nbx, blocks ? blocks->x_iface : nullptr);
  if (s == HZ_OK) s = build_axis(p->ay, grid->ny, grid->hy, nby, blocks ? blocks->y_iface : nullptr);
  p->need_global = (nbx > 1 || nby > 1);
  if (s == HZ_OK && p->need_global) {
    s = build_global(p->ax);
    if (s == HZ_OK) s = build_global(p->ay);
  }
  if (s == HZ_OK) {
    p->info.eig_max_residual = std::max(p->ax.eig_res, p->ay.eig_res);
    if (!(p->info.eig_max_residual < 1e-9)) s = HZ_ERR_EIG;
  }
  if (s != HZ_OK) { delete p; return s; }
  try {
    ck(cudaGetDevice(&p->device));
    ck(cudaDeviceGetAttribute(&p->sms, cudaDevAttrMultiProcessorCount, p->device));
    hz::dst_prepare(hz::kDstMaxN);
    ck(cudaStreamCreateWithFlags(&p->side, cudaStreamNonBlocking));
    ck(cudaEventCreateWithFlags(&p->ev_fork, cudaEventDisableTiming));
    ck(cudaEventCreateWithFlags(&p->ev_join, cudaEventDisableTiming));
    p->status = dalloc<int>(p, 1);
    p->minpiv = dalloc<unsigned long long>(p, 1);
    build_axis_dev(p, p->ax, p->dx, p->need_global);
    build_axis_dev(p, p->ay, p->dy, p->need_global);
    build_stencil_xy(p);
    build_z(p);
    ck(cudaStreamSynchronize(p->st));
  } catch (const Fail& e) {
    release(p);
    delete p;
    return e.s;
  }
  p->info.plan_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  p->info.device_bytes = p->bytes;
  *out = p;
  return HZ_OK;
}

hz_status hz_plan_set_frequency(hz_plan_t p, double omega) {
  if (!p || !std::isfinite(omega)) return HZ_ERR_ARG;
  const auto t0 = std::chrono::steady_clock::now();
  p->omega = omega;
  try {
    build_z(p);
  } catch (const Fail& e) {
    return e.s;
  }
  p->info.plan_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  return HZ_OK;
}

hz_status hz_plan_set_k2(hz_plan_t p, const hz_c128* k2) {
  if (!p || !k2) return HZ_ERR_ARG;
  for (int L = 0; L < p->nlayers; ++L)
    if (!std::isfinite(k2[L].re) || !std::isfinite(k2[L].im)) return HZ_ERR_ARG;
  const auto t0 = std::chrono::steady_clock::now();
  for (int L = 0; L < p->nlayers; ++L) p->k2base[L] = cd(k2[L].re, k2[L].im);
  try {
    build_z(p);
  } catch (const Fail& e) {
    return e.s;
  }
  p->info.plan_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  return HZ_OK;
}

hz_status hz_tridiag_eig(int n, const hz_c128* kd, const hz_c128* ko, const hz_c128* m, hz_c128* lam,
                         hz_c128* W, double* residual) {
  if (n < 1 || !kd || !m || !lam || !W || (n > 1 && !ko)) return HZ_ERR_ARG;
  std::vector<cd> d(n), o(std::max(n - 1, 1)), mm(n), l, w;
  for (int i = 0; i < n; ++i) {
    d[i] = cd(kd[i].re, kd[i].im);
    mm[i] = cd(m[i].re, m[i].im);
  }
  for (int i = 0; i + 1 < n; ++i) o[i] = cd(ko[i].re, ko[i].im);
  double res = 0.0;
  if (!hz::tridiag_eig(n, d.data(), o.data(), mm.data(), l, w, &res)) return HZ_ERR_EIG;
  for (int i = 0; i < n; ++i) lam[i] = hz_c128{l[i].real(), l[i].imag()};
  for (size_t i = 0; i < (size_t)n * n; ++i) W[i] = hz_c128{w[i].real(), w[i].imag()};
  if (residual) *residual = res;
  return HZ_OK;
}

hz_status hz_plan_set_fast_sine(hz_plan_t p, int enable) {
  if (!p || enable < 0 || enable > 2) return HZ_ERR_ARG;
  p->fast_sine = enable >= 1;
  p->fast_sine32 = enable == 2;
  return HZ_OK;
}

hz_status hz_plan_set_real_tables(hz_plan_t p, int enable) {
  if (!p) return HZ_ERR_ARG;
  p->tc_real = enable != 0;
  return HZ_OK;
}

hz_status hz_plan_set_dense_tile_rows(hz_plan_t p, int rows) {
  if (!p || (rows != 0 && rows != 16 && rows != 64)) return HZ_ERR_ARG;
  p->xf_tile = rows;
  return HZ_OK;
}

hz_status hz_plan_set_z_sweep(hz_plan_t p, int variant) {
  if (!p || variant < 0 || variant > 3) return HZ_ERR_ARG;
  p->zs_rb = variant;
  return HZ_OK;
}

hz_status hz_sine_transform_host(int n, int dir, double scale, const hz_c128* in, hz_c128* out) {
  if (n < 2 || !in || !out || (dir != 1 && dir != 2) || !std::isfinite(scale)) return HZ_ERR_ARG;
  if (!hz::dst_apply_host(n, dir, scale, reinterpret_cast<const double2*>(in), reinterpret_cast<double2*>(out)))
    return HZ_ERR_ARG;
  return HZ_OK;
}

hz_status hz_plan_set_options(hz_plan_t p, const hz_options* opts) {
  if (!p || !opts) return HZ_ERR_ARG;
  if (opts->precision < HZ_FP64 || opts->precision > HZ_MIXED_TF32) return HZ_ERR_ARG;
  p->opts = *opts;
  if (!(p->opts.rtol > 0)) p->opts.rtol = 1e-8;
  if (p->opts.max_refine < 0) p->opts.max_refine = 0;
  p->st = (cudaStream_t)opts->cuda_stream;
  return HZ_OK;
}

hz_status hz_solve(hz_plan_t p, const hz_c128* f, hz_c128* u, int nrhs) {
  if (!p || !f || !u || nrhs < 1) return HZ_ERR_ARG;
  try {
    solve_full(p, reinterpret_cast<const double2*>(f), reinterpret_cast<double2*>(u), nrhs, 0);
  } catch (const Fail& e) {
    return e.s;
  }
  return HZ_OK;
}

hz_status hz_solve_host(hz_plan_t p, const hz_c128* f, hz_c128* u, int nrhs) {
  if (!p || !f || !u || nrhs < 1) return HZ_ERR_ARG;
  try {
    ensure_ws(p, nrhs);
    const size_t per = (size_t)p->nx * p->ny * p->nz;          // complex values per RHS
    double2* fd = ensure_extra(p, p->ws.F2, p->ws.f2_cap, nrhs);
    double2* ud = ensure_extra(p, p->ws.HU, p->ws.hu_cap, nrhs);
    const double2* fh = reinterpret_cast<const double2*>(f);
    double2* uh = reinterpret_cast<double2*>(u);
    if (nrhs < 2) {
      ck(cudaMemcpyAsync(fd, fh, sizeof(double2) * per * nrhs, cudaMemcpyHostToDevice, p->st));
      solve_full(p, fd, ud, nrhs, 0);
      ck(cudaMemcpyAsync(uh, ud, sizeof(double2) * per * nrhs, cudaMemcpyDeviceToHost, p->st));
      ck(cudaStreamSynchronize(p->st));
    } else {
      // up to eight chunks of RHS: every upload is queued at once on one copy stream (chunk c's
      // solve waits for its own upload only), each chunk's download starts on a second copy
      // stream as soon as its solve is done, so both directions overlap the later solves
      if (!p->cst) {
        ck(cudaStreamCreateWithFlags(&p->cst, cudaStreamNonBlocking));
        ck(cudaStreamCreateWithFlags(&p->cst2, cudaStreamNonBlocking));
        for (cudaEvent_t& e : p->ev_in) ck(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
      }
      const int K = std::min(nrhs, 8);
      int r0[9];
      for (int c = 0; c <= K; ++c) r0[c] = (int)((long long)nrhs * c / K);
      for (int c = 0; c < K; ++c) {
        const size_t off = per * r0[c], bytes = sizeof(double2) * per * (r0[c + 1] - r0[c]);
        ck(cudaMemcpyAsync(fd + off, fh + off, bytes, cudaMemcpyHostToDevice, p->cst));
        ck(cudaEventRecord(p->ev_in[c], p->cst));
      }
      int refs = 0;
      double rel = -1.0;
      for (int c = 0; c < K; ++c) {
        const size_t off = per * r0[c], bytes = sizeof(double2) * per * (r0[c + 1] - r0[c]);
        ck(cudaStreamWaitEvent(p->st, p->ev_in[c], 0));
        solve_full(p, fd + off, ud + off, r0[c + 1] - r0[c], 0);   // returns with the solve done
        refs = std::max(refs, p->info.refinements);
        rel = std::max(rel, p->info.rel_residual);
        ck(cudaMemcpyAsync(uh + off, ud + off, bytes, cudaMemcpyDeviceToHost, p->cst2));
      }
      ck(cudaStreamSynchronize(p->st));
      ck(cudaStreamSynchronize(p->cst2));
      p->info.refinements = refs;
      p->info.rel_residual = rel;
    }
  } catch (const Fail& e) {
    if (p->cst) cudaStreamSynchronize(p->cst);             // no copy may touch the caller's buffers later
    if (p->cst2) cudaStreamSynchronize(p->cst2);
    return e.s;
  }
  return HZ_OK;
}

hz_status hz_solve_adjoint(hz_plan_t p, const hz_c128* g, hz_c128* lam, int nrhs) {
  if (!p || !g || !lam || nrhs < 1) return HZ_ERR_ARG;
  try {
    ensure_ws(p, nrhs);
    double2* f2 = ensure_extra(p, p->ws.F2, p->ws.f2_cap, nrhs);
    hz::adjoint_prep(reinterpret_cast<const double2*>(g), f2, p->dx.im, p->dy.im, p->imz, p->nx, p->ny,
                     p->nz, nrhs, p->st);
    solve_full(p, f2, reinterpret_cast<double2*>(lam), nrhs, 1);
  } catch (const Fail& e) {
    return e.s;
  }
  return HZ_OK;
}

}  // extern "C"

namespace {

// The GMRES of hz_solve_perturbed with a Krylov basis of element type VT: double2 (FP64
// plans) or float2 (mixed plans: the basis in complex64, combined in FP32 against FP64
// vectors; the restart residuals, the solves and the iterate stay FP64, so the restarts
// correct what the FP32 basis loses).
template <typename VT>
hz_status perturbed_impl(hz_plan_t p, const hz_c128* dk2_dev, const hz_c128* f_dev, hz_c128* u_dev, int nrhs,
                         double rtol, int max_iter, int restart, int* iters_out, double* relres_out) {
  using cplx = std::complex<double>;
  const int m = restart < 1 ? 20 : std::min(restart, 200);
  const int R = nrhs;
  const long long n = (long long)p->nx * p->ny * p->nz;
  const long long vol = n * R;
  std::vector<void*> mine;
  auto local = [&](size_t count) {
    double2* b = dalloc<double2>(p, count);
    mine.push_back(b);
    return b;
  };
  hz_status status = HZ_OK;
  int iters = 0;
  try {
    ensure_ws(p, R);
    cudaStream_t st = p->st;
    const double2* d = reinterpret_cast<const double2*>(dk2_dev);
    const double2* f = reinterpret_cast<const double2*>(f_dev);
    double2* X = reinterpret_cast<double2*>(u_dev);
    VT* V = dalloc<VT>(p, (size_t)(m + 1) * vol);            // Krylov basis [i][r][n]
    mine.push_back(V);
    double2* B = local(vol);                                // S f
    double2* T = local(vol);
    double2* Wv = local(vol);
    double2* partial = local((size_t)R * hz::multi_dot_parts(n) * hz::kMaxVec);
    double2* dots = local((size_t)R * hz::kMaxVec);
    double2* coef = local((size_t)R * hz::kMaxVec);
    double2* hd = local((size_t)(2 * (m + 1) + 1) * R);    // projections of one iteration + <w, w>
    std::vector<double2> hh((size_t)(2 * (m + 1) + 1) * R);
    std::vector<double2> hbuf((size_t)R * hz::kMaxVec);
    // <V_i, w> for i in [i0, i0 + cnt) -> host, [r][i]
    auto dot_host = [&](const double2* Vb, int cnt, const double2* w) {
      hz::multi_dot(Vb, vol, cnt, w, n, R, partial, dots, st);
      ck(cudaMemcpyAsync(hbuf.data(), dots, sizeof(double2) * R * cnt, cudaMemcpyDeviceToHost, st));
      ck(cudaStreamSynchronize(st));
      std::vector<cplx> out((size_t)R * cnt);
      for (int q = 0; q < R * cnt; ++q) out[q] = cplx(hbuf[q].x, hbuf[q].y);
      return out;
    };
    auto axpy_host = [&](const VT* Vb, int cnt, const std::vector<cplx>& c, double2* w) {   // w -= V c
      for (int q = 0; q < R * cnt; ++q) hbuf[q] = make_double2(c[q].real(), c[q].imag());
      ck(cudaMemcpyAsync(coef, hbuf.data(), sizeof(double2) * R * cnt, cudaMemcpyHostToDevice, st));
      hz::multi_axpy(Vb, vol, cnt, coef, w, n, R, st);
    };
    auto norms = [&](const double2* w) {
      const std::vector<cplx> q = dot_host(w, 1, w);
      std::vector<double> o(R);
      for (int r = 0; r < R; ++r) o[r] = std::sqrt(std::max(q[r].real(), 0.0));
      return o;
    };
    auto scale_into = [&](const std::vector<double>& s, const double2* w, VT* out) {
      for (int r = 0; r < R; ++r) hbuf[r] = make_double2(s[r], 0.0);
      ck(cudaMemcpyAsync(coef, hbuf.data(), sizeof(double2) * R, cudaMemcpyHostToDevice, st));
      hz::vec_scale(coef, w, out, n, R, st);
    };

    solve_full(p, f, B, R, 0);                              // right-hand side S f
    ck(cudaMemcpyAsync(X, B, sizeof(double2) * vol, cudaMemcpyDeviceToDevice, st));   // Born guess
    const std::vector<double> bnorm = norms(B);
    std::vector<cplx> H((size_t)R * (m + 1) * m), g((size_t)R * (m + 1)), cs((size_t)R * m), sn((size_t)R * m);
    auto Hat = [&](int r, int i, int j) -> cplx& { return H[((size_t)r * (m + 1) + i) * m + j]; };
    bool conv = false;
    while (!conv && iters < max_iter) {
      // r0 = B - L(X) = B - X + S(dk2 X)
      hz::pert_mul(d, X, T, n, R, st);
      solve_full(p, T, Wv, R, 0);
      hz::vec_lin3(B, X, Wv, T, vol, st);
      const std::vector<double> beta = norms(T);
      conv = true;
      for (int r = 0; r < R; ++r) conv = conv && beta[r] <= rtol * bnorm[r];
      if (conv) break;
      std::vector<double> inv(R);
      for (int r = 0; r < R; ++r) inv[r] = beta[r] > 0.0 ? 1.0 / beta[r] : 0.0;
      scale_into(inv, T, V);
      std::fill(H.begin(), H.end(), cplx(0));
      std::fill(g.begin(), g.end(), cplx(0));
      for (int r = 0; r < R; ++r) g[(size_t)r * (m + 1)] = beta[r];
      int j = 0;
      while (j < m && iters < max_iter) {
        // Arnoldi on K = S dk2 (L = I - K has the same Krylov space; its Hessenberg matrix is
        // I - H_K): K v_j carries no large component along v_j, so one Gram-Schmidt pass is
        // usually enough
        VT* Vj = V + (size_t)j * vol;
        hz::pert_mul(d, Vj, T, n, R, st);
        solve_full(p, T, Wv, R, 0);
        ++iters;
        // classical Gram-Schmidt in chunks of kMaxVec basis vectors, the projections kept on
        // the device (hd[pass][i][r]); a second pass only when the first one cancelled most
        // of the vector (||w after|| < ||w before|| / sqrt(2), the DGKS test, with
        // ||w before||^2 = ||w after||^2 + sum |h|^2).  On GB300 every pass is bound by the
        // FP64 pipe (4 FMA per complex element and basis vector), so the test saves half.
        double2* nn = hd + (size_t)2 * (m + 1) * R;        // <w, w> per RHS
        auto project = [&](int pass) {
          for (int i0 = 0; i0 <= j; i0 += hz::kMaxVec) {
            const int cnt = std::min(hz::kMaxVec, j + 1 - i0);
            double2* hc = hd + ((size_t)pass * (m + 1) + i0) * R;
            hz::multi_dot(V + (size_t)i0 * vol, vol, cnt, Wv, n, R, partial, hc, st);
            hz::multi_axpy(V + (size_t)i0 * vol, vol, cnt, hc, Wv, n, R, st);
          }
          hz::multi_dot(Wv, vol, 1, Wv, n, R, partial, nn, st);
          ck(cudaMemcpyAsync(hh.data(), hd, sizeof(double2) * hh.size(), cudaMemcpyDeviceToHost, st));
          ck(cudaStreamSynchronize(st));
          double worst = 1.0;                                 // min over RHS of after^2 / before^2
          for (int r = 0; r < R; ++r) {
            double hs = 0.0;
            for (int i0 = 0; i0 <= j; i0 += hz::kMaxVec) {
              const int cnt = std::min(hz::kMaxVec, j + 1 - i0);
              const double2* hc = hh.data() + ((size_t)pass * (m + 1) + i0) * R;
              for (int i = 0; i < cnt; ++i) {
                const cplx h(hc[r * cnt + i].x, hc[r * cnt + i].y);
                Hat(r, i0 + i, j) -= h;                    // H_L = I - H_K
                hs += std::norm(h);
              }
            }
            const double after = std::max(hh[(size_t)2 * (m + 1) * R + r].x, 0.0);
            if (after + hs > 0.0) worst = std::min(worst, after / (after + hs));
          }
          return worst;
        };
        for (int r = 0; r < R; ++r) Hat(r, j, j) += 1.0;
        if (project(0) < 0.5) project(1);
        hz::vec_inv_norm(nn, coef, R, st);
        hz::vec_scale(coef, Wv, V + (size_t)(j + 1) * vol, n, R, st);
        for (int r = 0; r < R; ++r)
          Hat(r, j + 1, j) = -std::sqrt(std::max(hh[(size_t)2 * (m + 1) * R + r].x, 0.0));
        // Givens rotations G = [[c, s], [-conj(s), c]], c real
        bool all = true;
        for (int r = 0; r < R; ++r) {
          for (int i = 0; i < j; ++i) {
            const cplx c = cs[(size_t)r * m + i], sv = sn[(size_t)r * m + i];
            const cplx a = Hat(r, i, j), b = Hat(r, i + 1, j);
            Hat(r, i, j) = c * a + sv * b;
            Hat(r, i + 1, j) = -std::conj(sv) * a + c * b;
          }
          const cplx a = Hat(r, j, j), b = Hat(r, j + 1, j);
          const double t = std::sqrt(std::norm(a) + std::norm(b));
          cplx c = 1.0, sv = 0.0;
          if (t > 0.0) {
            if (std::abs(a) == 0.0) { c = 0.0; sv = 1.0; }
            else { c = std::abs(a) / t; sv = (a / std::abs(a)) * std::conj(b) / t; }
          }
          cs[(size_t)r * m + j] = c;
          sn[(size_t)r * m + j] = sv;
          Hat(r, j, j) = c * a + sv * b;
          Hat(r, j + 1, j) = 0.0;
          const cplx gj = g[(size_t)r * (m + 1) + j];
          g[(size_t)r * (m + 1) + j] = c * gj;
          g[(size_t)r * (m + 1) + j + 1] = -std::conj(sv) * gj;
          all = all && std::abs(g[(size_t)r * (m + 1) + j + 1]) <= rtol * bnorm[r];
        }
        ++j;
        if (all) break;
      }
      // X += V y with H y = g (upper triangular, j x j), per RHS
      std::vector<cplx> y((size_t)R * j, cplx(0));
      for (int r = 0; r < R; ++r)
        for (int i = j - 1; i >= 0; --i) {
          cplx acc = g[(size_t)r * (m + 1) + i];
          for (int k = i + 1; k < j; ++k) acc -= Hat(r, i, k) * y[(size_t)r * j + k];
          const cplx hii = Hat(r, i, i);
          y[(size_t)r * j + i] = std::abs(hii) > 0.0 ? acc / hii : cplx(0);
        }
      for (int i0 = 0; i0 < j; i0 += hz::kMaxVec) {
        const int cnt = std::min(hz::kMaxVec, j - i0);
        std::vector<cplx> c((size_t)R * cnt);
        for (int r = 0; r < R; ++r)
          for (int i = 0; i < cnt; ++i) c[(size_t)r * cnt + i] = -y[(size_t)r * j + i0 + i];
        axpy_host(V + (size_t)i0 * vol, cnt, c, X);
      }
    }
    // true residual of the perturbed operator: ||M (f + dk2 u) - A u|| / ||M f||
    std::vector<double> fn2, rel;
    residual_core(p, f, X, nullptr, R, nullptr, fn2);      // caches ||M f||^2 per RHS
    hz::pert_mul(d, X, T, n, R, st);
    hz::vec_lin3(f, nullptr, T, T, vol, st);
    residual_core(p, T, X, nullptr, R, &rel, fn2);
    if (relres_out)
      for (int r = 0; r < R; ++r) relres_out[r] = rel[r];
    if (!conv) status = HZ_ERR_NOT_CONVERGED;
  } catch (const Fail& e) {
    status = e.s;
  }
  cudaStreamSynchronize(p->st);
  for (void* b : mine) dfree(p, b);
  if (iters_out) *iters_out = iters;
  return status;
}

}  // namespace

extern "C" {

hz_status hz_solve_perturbed(hz_plan_t p, const hz_c128* dk2_dev, const hz_c128* f_dev, hz_c128* u_dev, int nrhs,
                             double rtol, int max_iter, int restart, int* iters_out, double* relres_out) {
  if (!p || !dk2_dev || !f_dev || !u_dev || nrhs < 1 || !(rtol > 0.0) || max_iter < 1) return HZ_ERR_ARG;
  if (static_cast<const void*>(f_dev) == static_cast<const void*>(u_dev)) return HZ_ERR_ARG;
  if (p->opts.precision != HZ_FP64)
    return perturbed_impl<float2>(p, dk2_dev, f_dev, u_dev, nrhs, rtol, max_iter, restart, iters_out, relres_out);
  return perturbed_impl<double2>(p, dk2_dev, f_dev, u_dev, nrhs, rtol, max_iter, restart, iters_out, relres_out);
}


hz_status hz_grad_layers(hz_plan_t p, const hz_c128* u, const hz_c128* lam, int nrhs, hz_c128* G_host) {
  if (!p || !u || !lam || !G_host || nrhs < 1) return HZ_ERR_ARG;
  NvtxRange range("hz layer gradient");
  try {
    Workspace& w = p->ws;
    const int parts = hz::grad_parts(p->nx, p->ny, nrhs);
    dfree(p, w.gpart);
    dfree(p, w.Gl);
    w.gpart = dalloc<double2>(p, (size_t)parts * p->nz);
    w.Gl = dalloc<double2>(p, p->nlayers);
    hz::grad_layers(reinterpret_cast<const double2*>(u), reinterpret_cast<const double2*>(lam), p->dx.m,
                    p->dy.m, p->mz, p->zb, p->nlayers, p->nx, p->ny, p->nz, nrhs, w.gpart, parts, w.Gl,
                    p->st);
    ck(cudaGetLastError());
    ck(cudaMemcpyAsync(G_host, w.Gl, sizeof(double2) * p->nlayers, cudaMemcpyDeviceToHost, p->st));
    ck(cudaStreamSynchronize(p->st));
  } catch (const Fail& e) {
    return e.s;
  }
  return HZ_OK;
}

hz_status hz_grad_rhs(hz_plan_t p, const hz_c128* lam, hz_c128* gf, int nrhs) {
  if (!p || !lam || !gf || nrhs < 1) return HZ_ERR_ARG;
  NvtxRange range("hz right-hand-side gradient");
  try {
    hz::grad_rhs(reinterpret_cast<const double2*>(lam), reinterpret_cast<double2*>(gf), p->dx.m, p->dy.m, p->mz,
                 p->nx, p->ny, p->nz, nrhs, p->st);
    ck(cudaGetLastError());
    ck(cudaStreamSynchronize(p->st));
  } catch (const Fail& e) {
    return e.s;
  }
  return HZ_OK;
}

hz_status hz_residual(hz_plan_t p, const hz_c128* f, const hz_c128* u, int nrhs, double* rel_host) {
  if (!p || !f || !u || !rel_host || nrhs < 1) return HZ_ERR_ARG;
  try {
    ensure_ws(p, nrhs);
    double2* rho = ensure_extra(p, p->ws.RHO, p->ws.rho_cap, nrhs);
    std::vector<double> rel, fn2;
    residual_core(p, reinterpret_cast<const double2*>(f), reinterpret_cast<const double2*>(u), nullptr, nrhs,
                  &rel, fn2);
    (void)rho;
    for (int r = 0; r < nrhs; ++r) rel_host[r] = rel[r];
  } catch (const Fail& e) {
    return e.s;
  }
  return HZ_OK;
}

hz_status hz_set_stage_timing(hz_plan_t p, int enable) {
  if (!p) return HZ_ERR_ARG;
  if (cudaStreamSynchronize(p->st) != cudaSuccess) return HZ_ERR_CUDA;
  collect_stages(p);
  p->timing = enable != 0;
  for (int s = 0; s < HZ_NSTAGES; ++s) {
    p->stage_ms[s] = 0.0;
    p->stage_launches[s] = 0;
  }
  return HZ_OK;
}

hz_status hz_get_stage_times(hz_plan_t p, double* ms, long long* launches) {
  if (!p) return HZ_ERR_ARG;
  for (int s = 0; s < HZ_NSTAGES; ++s) {
    if (ms) ms[s] = p->stage_ms[s];
    if (launches) launches[s] = p->stage_launches[s];
  }
  return HZ_OK;
}

hz_status hz_get_info(hz_plan_t p, hz_info* out) {
  if (!p || !out) return HZ_ERR_ARG;
  p->info.device_bytes = p->bytes;
  p->info.tensor_cores = p->use_tc ? 1 : 0;
  p->info.fast_sine = p->has_dst ? (p->fast_sine32 ? 2 : (p->fast_sine ? 1 : 0)) : 0;
  p->info.real_tables = (p->tc_real && p->has_real_tc) ? 1 : 0;
  p->info.z_sweep = p->zs_rb;
  *out = p->info;
  return HZ_OK;
}

hz_status hz_plan_autotune(hz_plan_t p, int nrhs, int* choice_out) {
  if (!p || nrhs < 1) return HZ_ERR_ARG;
  try {
    ensure_ws(p, nrhs);
    double2* buf = ensure_extra(p, p->ws.F2, p->ws.f2_cap, nrhs);
    double2* out = ensure_extra(p, p->ws.HU, p->ws.hu_cap, nrhs);
    ck(cudaMemsetAsync(buf, 0, sizeof(double2) * (size_t)p->nx * p->ny * p->nz * nrhs, p->st));
    const int c = tune_plan(p, p->ws, p->st, buf, out, nrhs);
    if (choice_out) *choice_out = c;
  } catch (const Fail& e) {
    return e.s;
  }
  return HZ_OK;
}

hz_status hz_batch_create(int nitems, const hz_plan_t* plans, const int* nrhs, int nlanes, hz_batch_t* out) {
  if (!out) return HZ_ERR_ARG;
  *out = nullptr;
  if (nitems < 1 || !plans || !nrhs || nlanes < 0) return HZ_ERR_ARG;
  for (int i = 0; i < nitems; ++i)
    if (!plans[i] || nrhs[i] < 1) return HZ_ERR_ARG;
  for (int i = 0; i < nitems; ++i)
    for (int j = 0; j < i; ++j)
      if (plans[i] == plans[j]) return HZ_ERR_ARG;      // a plan's status word is per item
  hz_batch_t b = new (std::nothrow) hz_batch_s();
  if (!b) return HZ_ERR_OOM;
  b->plans.assign(plans, plans + nitems);
  b->nrhs.assign(nrhs, nrhs + nitems);
  try {
    hz::xform_tc_prepare();
    batch_setup(b, nlanes == 0 ? 4 : nlanes);
  } catch (const Fail& e) {
    bfree(b);
    delete b;
    return e.s;
  }
  *out = b;
  return HZ_OK;
}

hz_status hz_batch_solve(hz_batch_t b, const hz_c128* const* f_dev, hz_c128* const* u_dev, double* rel_host) {
  if (!b || !f_dev || !u_dev) return HZ_ERR_ARG;
  for (size_t i = 0; i < b->plans.size(); ++i)
    if (!f_dev[i] || !u_dev[i] || f_dev[i] == u_dev[i]) return HZ_ERR_ARG;
  try {
    batch_run(b, f_dev, u_dev, rel_host);
  } catch (const Fail& e) {
    return e.s;
  }
  return HZ_OK;
}

hz_status hz_batch_autotune(hz_batch_t b, const hz_c128* const* f_dev, hz_c128* const* u_dev, int* lanes_out) {
  if (!b || !f_dev || !u_dev) return HZ_ERR_ARG;
  try {
    const int n = (int)b->plans.size();
    // tune every plan on the batch's own lane workspace (one lane: sized for the largest
    // item) and the caller's buffers, so that no plan allocates a workspace of its own
    batch_setup(b, 1);
    for (int i = 0; i < n; ++i)
      tune_plan(b->plans[i], b->ws[0], b->s0, reinterpret_cast<const double2*>(f_dev[i]),
                reinterpret_cast<double2*>(u_dev[i]), b->nrhs[i]);
    int best_l = b->nlanes;
    double best_ms = 1e300;
    for (int l : {1, 2, 4, 8}) {
      if (l > n) break;
      batch_setup(b, l);
      batch_run(b, f_dev, u_dev, nullptr);                 // capture + first replay
      double ms = 0.0;
      for (int rep = 0; rep < 2; ++rep) {
        batch_run(b, f_dev, u_dev, nullptr);
        ms += b->last_ms;
      }
      if (ms < best_ms) { best_ms = ms; best_l = l; }
    }
    batch_setup(b, best_l);
    if (lanes_out) *lanes_out = best_l;
  } catch (const Fail& e) {
    return e.s;
  }
  return HZ_OK;
}

hz_status hz_batch_info(hz_batch_t b, double* last_ms, long long* launches_per_replay, int* lanes) {
  if (!b) return HZ_ERR_ARG;
  if (last_ms) *last_ms = b->last_ms;
  if (launches_per_replay) *launches_per_replay = b->launches_per_replay;
  if (lanes) *lanes = b->nlanes;
  return HZ_OK;
}

hz_status hz_batch_destroy(hz_batch_t b) {
  if (!b) return HZ_ERR_ARG;
  if (b->s0) cudaStreamSynchronize(b->s0);
  bfree(b);
  delete b;
  return HZ_OK;
}

hz_status hz_plan_destroy(hz_plan_t p) {
  if (!p) return HZ_ERR_ARG;
  cudaStreamSynchronize(p->st);
  release(p);
  delete p;
  return HZ_OK;
}

}  // extern "C"
