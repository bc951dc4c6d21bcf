// igks_api.cu -- host side of libigks: the C ABI of include/igks.h.
//
// Holds the contexts, validates and lays out the meshes of all solves of a context in
// one set of device buffers, builds the LU-SGS level schedule (cells grouped by their
// depth in the dependency graph of the sequential sweep of Eq. 20), captures one
// iteration as a CUDA graph and replays it, and copies fields in and out.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/igks.h"
#include "igks_dev.h"

using namespace igks;

// last error of the context-free entry point (igks_noalloc.cu)
const char* igks_noalloc_last_error_();

namespace {

struct HostMesh {
  int nn = 0, nc = 0, nf = 0;
  std::vector<double> xy;
  std::vector<int> cell_ptr, cell_nodes, face_nodes, face_cells, face_bc;
  int nlev_f = 0, nlev_b = 0, nbf = 0;
};

struct Buf {
  void* p = nullptr;
  size_t bytes = 0;
};

}  // namespace

struct igks_ctx {
  igks_options opt{};
  std::vector<HostMesh> meshes;
  std::vector<igks_flow> flows;
  std::vector<int> flow_set;
  bool built = false;
  Dev dev{};
  std::vector<Buf> bufs;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  std::string err = "";
  // layout
  std::vector<int> cell_off, cell_pad, face_off, node_off;
  SolveState* h_st = nullptr;   // pinned mirror of the per-solve state
  int nc_pad = 0, nf = 0, nn = 0;
  std::vector<int> h_wfwd_ptr, h_wbwd_ptr;   // wide schedule level offsets (host copies)
  // groups of consecutive solves, each iterated on a stream of its own (one group: the
  // context stream); per group its launch ranges, stream, graph and timing events
  int n_groups = 1;
  std::vector<Dev> gdev;
  std::vector<cudaStream_t> gstream;
  std::vector<cudaGraph_t> ggraph;
  std::vector<cudaGraphExec_t> ggexec;
  // the whole batch for check_every iterations as one graph: every group's chain of
  // iterations as a branch between a fork and a join (one launch per status check)
  cudaGraph_t bgraph = nullptr;
  cudaGraphExec_t bexec = nullptr;
  int bgraph_iters = 0;
  std::vector<std::vector<cudaEvent_t>> gev;
  std::vector<cudaEvent_t> join_ev;
  cudaEvent_t fork_ev = nullptr;
};

static int fail(igks_ctx* c, int code, const std::string& msg) {
  if (c) c->err = msg;
  return code;
}

#define CK(call)                                                                         \
  do {                                                                                   \
    cudaError_t e_ = (call);                                                             \
    if (e_ != cudaSuccess)                                                               \
      return fail(ctx, e_ == cudaErrorMemoryAllocation ? IGKS_ENOMEM : IGKS_ECUDA,       \
                  std::string(#call) + ": " + cudaGetErrorString(e_));                   \
  } while (0)


// every copy goes through the context stream (it does not synchronise with the legacy
// default stream); device-to-host copies wait for their data
static cudaError_t h2d(igks_ctx* c, void* dst, const void* src, size_t n) {
  return cudaMemcpyAsync(dst, src, n, cudaMemcpyHostToDevice, c->stream);
}
static cudaError_t d2h(igks_ctx* c, void* dst, const void* src, size_t n) {
  cudaError_t e = cudaMemcpyAsync(dst, src, n, cudaMemcpyDeviceToHost, c->stream);
  return e != cudaSuccess ? e : cudaStreamSynchronize(c->stream);
}
static cudaError_t h2d_2d(igks_ctx* c, void* dst, size_t dpitch, const void* src, size_t spitch, size_t w, size_t h) {
  return cudaMemcpy2DAsync(dst, dpitch, src, spitch, w, h, cudaMemcpyHostToDevice, c->stream);
}
static cudaError_t d2h_2d(igks_ctx* c, void* dst, size_t dpitch, const void* src, size_t spitch, size_t w, size_t h) {
  cudaError_t e = cudaMemcpy2DAsync(dst, dpitch, src, spitch, w, h, cudaMemcpyDeviceToHost, c->stream);
  return e != cudaSuccess ? e : cudaStreamSynchronize(c->stream);
}

static igks_flow default_flow() {
  igks_flow f{};
  f.mach = 0.15; f.reynolds = 1e5; f.aoa_deg = 0.0; f.prandtl = 0.72;
  f.t_ref = 288.15; f.s_suth = 110.4; f.sa_on = 0; f.limiter = 0; f.nut_ratio_inf = 3.0;
  f.cfl_exp = 1.0; f.cfl_init = 100.0; f.cfl_min = 100.0; f.cfl_max = 100.0;
  f.res_target = 1e-10; f.venkat_k = 5.0; f.c_num = 1.0; f.visc_sr = 0; f.eq40_target = 0.0;
  return f;
}

static DevFlow make_devflow(const igks_flow& f) {
  DevFlow d{};
  const double g = GAMMA;
  d.mach = f.mach; d.re = f.reynolds; d.prandtl = f.prandtl;
  d.s_star = f.s_suth / f.t_ref;
  d.lam_inf = g * f.mach * f.mach / 2.0;
  d.mu_inf = 1.0 / f.reynolds;
  d.nut_inf = f.sa_on ? f.nut_ratio_inf / f.reynolds : 0.0;
  d.p_inf = 1.0 / (g * f.mach * f.mach);
  double a = f.aoa_deg * M_PI / 180.0;
  double u = std::cos(a), v = std::sin(a);
  d.Winf[0] = 1.0; d.Winf[1] = u; d.Winf[2] = v;
  d.Winf[3] = d.p_inf / (g - 1.0) + 0.5 * (u * u + v * v);
  d.Winf[4] = d.nut_inf;
  d.cfl_exp = f.cfl_exp; d.cfl_init = f.cfl_init; d.cfl_min = f.cfl_min; d.cfl_max = f.cfl_max;
  d.res_target = f.res_target; d.venkat_k = f.venkat_k; d.c_num = f.c_num;
  d.eq40_target = f.eq40_target;
  d.pr_fix = 1.0 / f.prandtl - 1.0;
  d.sa_on = f.sa_on; d.limiter = f.limiter; d.visc_sr = f.visc_sr; d.scheme = f.scheme;
  return d;
}

template <class T>
static int dalloc(igks_ctx* ctx, T** out, size_t n) {
  void* p = nullptr;
  size_t bytes = std::max<size_t>(n, 1) * sizeof(T);
  CK(cudaMalloc(&p, bytes));
  CK(cudaMemsetAsync(p, 0, bytes, ctx->stream));
  ctx->bufs.push_back({p, bytes});
  *out = (T*)p;
  return 0;
}

template <class T>
static int upload(igks_ctx* ctx, const T** out, const std::vector<T>& h) {
  T* p;
  int rc = dalloc(ctx, &p, h.size());
  if (rc) return rc;
  if (!h.empty()) CK(h2d(ctx, p, h.data(), h.size() * sizeof(T)));
  *out = p;
  return 0;
}

// the per-group streams, graphs and events (group 0's stream is the context stream when
// there is one group)
static void release_groups(igks_ctx* ctx) {
  if (ctx->bexec) cudaGraphExecDestroy(ctx->bexec);
  if (ctx->bgraph) cudaGraphDestroy(ctx->bgraph);
  ctx->bexec = nullptr;
  ctx->bgraph = nullptr;
  ctx->bgraph_iters = 0;
  for (auto& g : ctx->ggexec) if (g) cudaGraphExecDestroy(g);
  for (auto& g : ctx->ggraph) if (g) cudaGraphDestroy(g);
  ctx->ggexec.clear();
  ctx->ggraph.clear();
  for (auto& evs : ctx->gev)
    for (auto e : evs) if (e) cudaEventDestroy(e);
  ctx->gev.clear();
  for (auto e : ctx->join_ev) if (e) cudaEventDestroy(e);
  ctx->join_ev.clear();
  if (ctx->fork_ev) cudaEventDestroy(ctx->fork_ev);
  ctx->fork_ev = nullptr;
  for (auto st : ctx->gstream)
    if (st && st != ctx->stream) cudaStreamDestroy(st);
  ctx->gstream.clear();
  ctx->gdev.clear();
}

static void release(igks_ctx* ctx) {
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  for (auto st : ctx->gstream) if (st) cudaStreamSynchronize(st);
  release_groups(ctx);
  for (auto& b : ctx->bufs) cudaFree(b.p);
  ctx->bufs.clear();
  if (ctx->h_st) cudaFreeHost(ctx->h_st);
  ctx->h_st = nullptr;
  ctx->built = false;
}

static const char* const KERNEL_NAMES[N_KERNEL_KINDS] = {
    "k_prep", "k_ghost", "k_gradient", "k_flux", "k_residual", "k_norms",
    "k_sweep_prep", "k_sweep_fwd", "k_sweep_bwd", "k_update", "k_end_iter"};

// issue one iteration's kernels of group g on its stream (with an event after each kernel
// when timing is on; event k+1 minus event k is the duration of kernel k)
static void enqueue_iteration(igks_ctx* ctx, int g) {
  const Dev& d = ctx->gdev[g];
  cudaStream_t s = ctx->gstream[g];
  const int p = ctx->opt.precision, th = ctx->opt.sweep_threads;
  const bool t = ctx->opt.timing != 0;
  cudaEvent_t* ev = t ? ctx->gev[g].data() : nullptr;
  int e = 0;
  if (t) cudaEventRecordWithFlags(ev[e++], s, cudaEventRecordExternal);
  launch_prep(d, s);                   if (t) cudaEventRecordWithFlags(ev[e++], s, cudaEventRecordExternal);
  launch_ghost(d, s);                  if (t) cudaEventRecordWithFlags(ev[e++], s, cudaEventRecordExternal);
  launch_gradient(d, s);               if (t) cudaEventRecordWithFlags(ev[e++], s, cudaEventRecordExternal);
  launch_flux(d, s);                   if (t) cudaEventRecordWithFlags(ev[e++], s, cudaEventRecordExternal);
  launch_residual(d, s);               if (t) cudaEventRecordWithFlags(ev[e++], s, cudaEventRecordExternal);
  launch_norms(d, s);                  if (t) cudaEventRecordWithFlags(ev[e++], s, cudaEventRecordExternal);
  launch_sweep_prep(d, p, s);          if (t) cudaEventRecordWithFlags(ev[e++], s, cudaEventRecordExternal);
  launch_sweep_fwd(d, p, th, s);       if (t) cudaEventRecordWithFlags(ev[e++], s, cudaEventRecordExternal);
  launch_sweep_bwd(d, p, th, s);       if (t) cudaEventRecordWithFlags(ev[e++], s, cudaEventRecordExternal);
  launch_update(d, p, s);              if (t) cudaEventRecordWithFlags(ev[e++], s, cudaEventRecordExternal);
  launch_end_iter(d, s);               if (t) cudaEventRecordWithFlags(ev[e++], s, cudaEventRecordExternal);
}

// the whole context as one launch range
static void whole_range(Dev& d) {
  d.g_blk0 = 0; d.g_nblk = d.n_cell_blocks;
  d.g_face0 = 0; d.g_nface = d.nf;
  d.g_solve0 = 0; d.g_nsolve = d.n_solves;
}

// Split the solves into groups of consecutive solves with about equal cell counts (one
// group with the wide schedule, whose per-level launches span all solves), give each its
// launch ranges, a stream and timing events, and capture one iteration of each as a graph.
static int setup_groups(igks_ctx* ctx) {
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  for (auto st : ctx->gstream) if (st) cudaStreamSynchronize(st);
  release_groups(ctx);
  Dev& d = ctx->dev;
  whole_range(d);
  const int ns = d.n_solves;
  int G = std::max(1, std::min(ctx->opt.groups, ns));
  if (d.wide) G = 1;
  ctx->n_groups = G;
  std::vector<int> cut(1, 0);
  {
    int64_t total = 0, acc = 0;
    for (int s = 0; s < ns; s++) total += ctx->cell_pad[s];
    for (int s = 0; s < ns && (int)cut.size() < G; s++) {
      acc += ctx->cell_pad[s];
      if (acc * G >= total * (int64_t)cut.size() && ns - (s + 1) >= G - (int)cut.size()) cut.push_back(s + 1);
    }
    while ((int)cut.size() < G) cut.push_back(cut.back() + 1);
    cut.push_back(ns);
  }
  for (int g = 0; g < G; g++) {
    Dev v = d;
    const int s0 = cut[g], s1 = cut[g + 1];
    v.g_solve0 = s0; v.g_nsolve = s1 - s0;
    v.g_blk0 = ctx->cell_off[s0] / CELL_BLOCK;
    v.g_nblk = (s1 < ns ? ctx->cell_off[s1] : ctx->nc_pad) / CELL_BLOCK - v.g_blk0;
    v.g_face0 = ctx->face_off[s0];
    v.g_nface = (s1 < ns ? ctx->face_off[s1] : ctx->nf) - v.g_face0;
    ctx->gdev.push_back(v);
    cudaStream_t st = ctx->stream;
    if (G > 1) CK(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    ctx->gstream.push_back(st);
    std::vector<cudaEvent_t> evs(N_KERNEL_KINDS + 1, nullptr);
    if (ctx->opt.timing)
      for (auto& e : evs) CK(cudaEventCreate(&e));
    ctx->gev.push_back(evs);
    cudaEvent_t j = nullptr;
    if (G > 1) CK(cudaEventCreateWithFlags(&j, cudaEventDisableTiming));
    ctx->join_ev.push_back(j);
  }
  if (G > 1) CK(cudaEventCreateWithFlags(&ctx->fork_ev, cudaEventDisableTiming));
  ctx->ggraph.assign(G, nullptr);
  ctx->ggexec.assign(G, nullptr);
  if (ctx->opt.use_graph) {
    for (int g = 0; g < G; g++) {
      CK(cudaStreamBeginCapture(ctx->gstream[g], cudaStreamCaptureModeThreadLocal));
      enqueue_iteration(ctx, g);
      cudaError_t e = cudaStreamEndCapture(ctx->gstream[g], &ctx->ggraph[g]);
      if (e != cudaSuccess) return fail(ctx, IGKS_ECUDA, std::string("graph capture: ") + cudaGetErrorString(e));
      CK(cudaGraphInstantiate(&ctx->ggexec[g], ctx->ggraph[g], 0));
    }
    // the batch graph: check_every iterations of every group, the groups' chains running
    // side by side (a group may run ahead of another inside it, as with the per-group
    // launches); not with per-kernel timing, whose events must stay one per kernel
    const int R = ctx->opt.check_every;
    if (!ctx->opt.timing && R >= 2 && R <= MAX_BATCH_GRAPH_ITERS) {
      CK(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
      if (G > 1) {
        cudaEventRecord(ctx->fork_ev, ctx->stream);
        for (int g = 0; g < G; g++) cudaStreamWaitEvent(ctx->gstream[g], ctx->fork_ev, 0);
      }
      for (int g = 0; g < G; g++)
        for (int r = 0; r < R; r++) enqueue_iteration(ctx, g);
      if (G > 1)
        for (int g = 0; g < G; g++) {
          cudaEventRecord(ctx->join_ev[g], ctx->gstream[g]);
          cudaStreamWaitEvent(ctx->stream, ctx->join_ev[g], 0);
        }
      cudaError_t e = cudaStreamEndCapture(ctx->stream, &ctx->bgraph);
      if (e != cudaSuccess) return fail(ctx, IGKS_ECUDA, std::string("batch graph capture: ") + cudaGetErrorString(e));
      CK(cudaGraphInstantiate(&ctx->bexec, ctx->bgraph, 0));
      ctx->bgraph_iters = R;
    }
  }
  return 0;
}

// n iterations of every group, stream-ordered after the work already on the context stream
// and before whatever the caller puts on it next
static int run_iterations(igks_ctx* ctx, int n) {
  const int G = ctx->n_groups;
  for (; ctx->bexec && n >= ctx->bgraph_iters; n -= ctx->bgraph_iters)   // whole check intervals
    CK(cudaGraphLaunch(ctx->bexec, ctx->stream));
  if (n == 0) {
    CK(cudaGetLastError());
    return 0;
  }
  if (G > 1) {
    CK(cudaEventRecord(ctx->fork_ev, ctx->stream));
    for (int g = 0; g < G; g++) CK(cudaStreamWaitEvent(ctx->gstream[g], ctx->fork_ev, 0));
  }
  for (int r = 0; r < n; r++)
    for (int g = 0; g < G; g++) {
      if (ctx->ggexec[g]) CK(cudaGraphLaunch(ctx->ggexec[g], ctx->gstream[g]));
      else enqueue_iteration(ctx, g);
    }
  if (G > 1) {
    for (int g = 0; g < G; g++) {
      CK(cudaEventRecord(ctx->join_ev[g], ctx->gstream[g]));
      CK(cudaStreamWaitEvent(ctx->stream, ctx->join_ev[g], 0));
    }
  }
  CK(cudaGetLastError());
  return 0;
}

// dependency levels of the sequential sweep: forward uses lower neighbours, backward upper
static void sweep_levels(const HostMesh& m, const std::vector<int>& cf_ptr, const std::vector<int>& cf_face,
                         bool forward, std::vector<int>& order, std::vector<int>& lvl_ptr) {
  const int n = m.nc;
  std::vector<int> lev(n, 0);
  int nlev = 0;
  for (int t = 0; t < n; t++) {
    int i = forward ? t : n - 1 - t;
    int L = 0;
    for (int k = cf_ptr[i]; k < cf_ptr[i + 1]; k++) {
      int f = cf_face[k];
      int l = m.face_cells[2 * f], r = m.face_cells[2 * f + 1];
      if (r < 0) continue;
      int j = (l == i) ? r : l;
      if (forward ? (j < i) : (j > i)) L = std::max(L, lev[j] + 1);
    }
    lev[i] = L;
    nlev = std::max(nlev, L + 1);
  }
  std::vector<int> cnt(nlev + 1, 0);
  for (int i = 0; i < n; i++) cnt[lev[i] + 1]++;
  for (int l = 0; l < nlev; l++) cnt[l + 1] += cnt[l];
  lvl_ptr.assign(cnt.begin(), cnt.end());
  order.assign(n, 0);
  std::vector<int> fill(cnt.begin(), cnt.end() - 1);
  for (int t = 0; t < n; t++) {
    int i = forward ? t : n - 1 - t;
    order[fill[lev[i]]++] = i;
  }
}

static int build(igks_ctx* ctx) {
  if (ctx->built) return 0;
  if (ctx->meshes.empty()) return fail(ctx, IGKS_EINVAL, "no mesh uploaded");
  const int ns = (int)ctx->meshes.size();
  CK(cudaSetDevice(ctx->opt.device));
  // ---- layout ----
  ctx->cell_off.assign(ns, 0); ctx->cell_pad.assign(ns, 0);
  ctx->face_off.assign(ns, 0); ctx->node_off.assign(ns, 0);
  int nc = 0, nf = 0, nn = 0;
  for (int s = 0; s < ns; s++) {
    const HostMesh& m = ctx->meshes[s];
    ctx->cell_off[s] = nc;
    ctx->cell_pad[s] = (m.nc + CELL_ALIGN - 1) / CELL_ALIGN * CELL_ALIGN;
    nc += ctx->cell_pad[s];
    ctx->face_off[s] = nf; nf += m.nf;
    ctx->node_off[s] = nn; nn += m.nn;
  }
  ctx->nc_pad = nc; ctx->nf = nf; ctx->nn = nn;
  std::vector<int> cell_solve(nc, -1), cf_ptr(nc + 1, 0), cf_face, cn_ptr(nc + 1, 0), cn_node;
  std::vector<double> xy(2 * (size_t)nn);
  std::vector<int> fL(nf), fR(nf), fbc(nf), fsolve(nf), fnode(2 * (size_t)nf), bface, wall_face, wall_ptr(ns + 1, 0);
  std::vector<int> fwd_order, fwd_lvl, bwd_order, bwd_lvl, lsp(ns + 1, 0), blsp(ns + 1, 0);
  std::vector<int> fs_ptr(1, 0), fs_j, fs_slot, cf_to_fs, bs_ptr(1, 0), bs_j, bs_slot, cf_to_bs;
  std::vector<SolveState> st(ns);
  std::vector<DevFlow> dfl(ns);
  for (int s = 0; s < ns; s++) {
    const HostMesh& m = ctx->meshes[s];
    const int co = ctx->cell_off[s], fo = ctx->face_off[s], no = ctx->node_off[s];
    for (int k = 0; k < m.nn; k++) {
      xy[no + k] = m.xy[2 * k];
      xy[nn + no + k] = m.xy[2 * k + 1];
    }
    // cell -> faces in ascending face order
    std::vector<int> lp(m.nc + 1, 0), lf;
    for (int f = 0; f < m.nf; f++) {
      lp[m.face_cells[2 * f] + 1]++;
      if (m.face_cells[2 * f + 1] >= 0) lp[m.face_cells[2 * f + 1] + 1]++;
    }
    for (int i = 0; i < m.nc; i++) lp[i + 1] += lp[i];
    lf.assign(lp[m.nc], 0);
    {
      std::vector<int> fill(m.nc, 0);
      for (int f = 0; f < m.nf; f++) {
        int l = m.face_cells[2 * f], r = m.face_cells[2 * f + 1];
        lf[lp[l] + fill[l]++] = f;
        if (r >= 0) lf[lp[r] + fill[r]++] = f;
      }
    }
    for (int i = 0; i < ctx->cell_pad[s]; i++) {
      int g = co + i;
      if (i < m.nc) {
        cell_solve[g] = s;
        for (int k = lp[i]; k < lp[i + 1]; k++) cf_face.push_back(fo + lf[k]);
        for (int k = m.cell_ptr[i]; k < m.cell_ptr[i + 1]; k++) cn_node.push_back(no + m.cell_nodes[k]);
      }
      cf_ptr[g + 1] = (int)cf_face.size();
      cn_ptr[g + 1] = (int)cn_node.size();
    }
    for (int f = 0; f < m.nf; f++) {
      int g = fo + f;
      fL[g] = co + m.face_cells[2 * f];
      fR[g] = m.face_cells[2 * f + 1] >= 0 ? co + m.face_cells[2 * f + 1] : -1;
      fbc[g] = m.face_bc[f];
      fsolve[g] = s;
      fnode[g] = no + m.face_nodes[2 * f];
      fnode[nf + g] = no + m.face_nodes[2 * f + 1];
      if (fR[g] < 0) bface.push_back(g);
      if (fR[g] < 0 && (fbc[g] == IGKS_BC_WALL || fbc[g] == IGKS_BC_MOVING_WALL)) wall_face.push_back(g);
    }
    wall_ptr[s + 1] = (int)wall_face.size();
    // sweep schedule
    std::vector<int> ord, lvl;
    sweep_levels(m, lp, lf, true, ord, lvl);
    ctx->meshes[s].nlev_f = (int)lvl.size() - 1;
    int base = (int)fwd_order.size();
    for (int c : ord) fwd_order.push_back(co + c);
    for (int p : lvl) fwd_lvl.push_back(base + p);
    lsp[s + 1] = (int)fwd_lvl.size();
    sweep_levels(m, lp, lf, false, ord, lvl);
    ctx->meshes[s].nlev_b = (int)lvl.size() - 1;
    base = (int)bwd_order.size();
    for (int c : ord) bwd_order.push_back(co + c);
    for (int p : lvl) bwd_lvl.push_back(base + p);
    blsp[s + 1] = (int)bwd_lvl.size();
    // narrow-schedule stencils in sweep-position order, with shared-memory ring slots: a
    // neighbour produced at position q is still in the ring while the current level (end
    // e) is processed iff q >= e - RING (no position written during the level maps to its
    // slot)
    cf_to_fs.resize(cf_face.size(), -1);
    cf_to_bs.resize(cf_face.size(), -1);
    for (int dir = 0; dir < 2; dir++) {
      const bool fwd = dir == 0;
      std::vector<int> ordl, lvll;
      sweep_levels(m, lp, lf, fwd, ordl, lvll);
      std::vector<int> pos(m.nc);
      for (int p = 0; p < m.nc; p++) pos[ordl[p]] = p;
      std::vector<int>& sptr = fwd ? fs_ptr : bs_ptr;
      std::vector<int>& sj = fwd ? fs_j : bs_j;
      std::vector<int>& sslot = fwd ? fs_slot : bs_slot;
      std::vector<int>& map = fwd ? cf_to_fs : cf_to_bs;
      for (int l = 0; l + 1 < (int)lvll.size(); l++) {
        const int e = lvll[l + 1];
        for (int p = lvll[l]; p < e; p++) {
          const int i = ordl[p];
          for (int k = lp[i]; k < lp[i + 1]; k++) {
            const int f = lf[k];
            const int l_ = m.face_cells[2 * f], r_ = m.face_cells[2 * f + 1];
            const int kg = cf_ptr[co + i] + (k - lp[i]);
            if (r_ < 0) {
              if (!fwd && (m.face_bc[f] == IGKS_BC_WALL || m.face_bc[f] == IGKS_BC_SYMMETRY ||
                           m.face_bc[f] == IGKS_BC_MOVING_WALL)) {
                map[kg] = (int)sj.size();
                sj.push_back(-1 - (fo + f));
                sslot.push_back(-1);
              }
              continue;
            }
            const int j = (l_ == i) ? r_ : l_;
            if (fwd ? (j >= i) : (j <= i)) continue;
            map[kg] = (int)sj.size();
            sj.push_back(co + j);
            sslot.push_back(pos[j] >= e - RING ? pos[j] % RING : -1);
          }
          sptr.push_back((int)sj.size());
        }
      }
    }
    // state
    SolveState& q = st[s];
    std::memset(&q, 0, sizeof q);
    q.cfl = ctx->flows[s].cfl_init;
    q.blk_begin = co / CELL_BLOCK;
    q.blk_end = (co + ctx->cell_pad[s]) / CELL_BLOCK;
    q.cell_begin = co;
    q.cell_end = co + m.nc;
    dfl[s] = make_devflow(ctx->flows[s]);
  }
  // ---- narrow schedule: per-position padded stencils (PF_E entries) and positions ----
  const int P = (int)fwd_order.size();
  std::vector<int> pos_f(nc, -1), pos_b(nc, -1);
  std::vector<FwdStat> fst(P);
  std::vector<BwdStat> bst(P);
  std::vector<int> cf_to_ef(cf_face.size(), -1), cf_to_eb(cf_face.size(), -1);
  for (int p = 0; p < P; p++) { pos_f[fwd_order[p]] = p; pos_b[bwd_order[p]] = p; }
  for (int p = 0; p < P; p++) {
    FwdStat& f = fst[p];
    BwdStat& b = bst[p];
    std::memset(&f, 0, sizeof f);
    std::memset(&b, 0, sizeof b);
    f.i = fwd_order[p]; f.pb = pos_b[fwd_order[p]];
    b.i = bwd_order[p];
    for (int e = 0; e < PF_E; e++) { f.slot[e] = -1; b.slot[e] = -1; }
  }
  for (int dir = 0; dir < 2; dir++) {
    const bool fwd = dir == 0;
    const std::vector<int>& sptr = fwd ? fs_ptr : bs_ptr;
    const std::vector<int>& sj = fwd ? fs_j : bs_j;
    const std::vector<int>& sslot = fwd ? fs_slot : bs_slot;
    const std::vector<int>& map = fwd ? cf_to_fs : cf_to_bs;
    std::vector<int>& emap = fwd ? cf_to_ef : cf_to_eb;
    std::vector<int> inv(sj.size(), -1);
    for (size_t k = 0; k < map.size(); k++)
      if (map[k] >= 0) inv[map[k]] = (int)k;
    for (int p = 0; p < P; p++) {
      int* cnt = fwd ? &fst[p].cnt : &bst[p].cnt;
      int* ej = fwd ? fst[p].j : bst[p].j;
      int* es = fwd ? fst[p].slot : bst[p].slot;
      const int q0 = sptr[p], m_ = sptr[p + 1] - q0;
      if (m_ > PF_E) { *cnt = -1; continue; }
      *cnt = m_;
      for (int e = 0; e < m_; e++) {
        ej[e] = sj[q0 + e];
        es[e] = sslot[q0 + e];
        emap[inv[q0 + e]] = p * PF_E + e;
      }
    }
  }
  // ---- device buffers ----
  Dev& d = ctx->dev;
  d = Dev{};
  d.n_solves = ns; d.nc_pad = nc; d.nf = nf; d.nn = nn; d.nbf = (int)bface.size();
  d.n_cell_blocks = nc / CELL_BLOCK;
  whole_range(d);
  int rc = 0;
#define UP(field, vec) if ((rc = upload(ctx, &d.field, vec))) { release(ctx); return rc; }
#define AL(field, type, n) if ((rc = dalloc(ctx, (type**)&d.field, n))) { release(ctx); return rc; }
  UP(xy, xy); UP(cell_solve, cell_solve); UP(cf_ptr, cf_ptr); UP(cf_face, cf_face);
  UP(cn_ptr, cn_ptr); UP(cn_node, cn_node);
  UP(fL, fL); UP(fR, fR); UP(fbc, fbc); UP(fsolve, fsolve); UP(fnode, fnode); UP(bface, bface);
  UP(wall_face, wall_face); UP(wall_ptr, wall_ptr);
  UP(fwd_order, fwd_order); UP(fwd_lvl, fwd_lvl); UP(bwd_order, bwd_order); UP(bwd_lvl, bwd_lvl);
  UP(lvl_solve_ptr, lsp); UP(blvl_solve_ptr, blsp); UP(flow, dfl);
  AL(area, double, nc); AL(cx, double, nc); AL(cy, double, nc); AL(wall_d, double, nc);
  AL(W, double, 5 * (size_t)nc); AL(grad, double, 8 * (size_t)nc); AL(phi, double, 4 * (size_t)nc);
  AL(omega, double, nc); AL(mu_l, double, nc); AL(mu_t, double, nc); AL(Lam, double, nc);
  AL(pu, double, nc); AL(pv, double, nc); AL(pc, double, nc); AL(lsq, double, 4 * (size_t)nc);
  AL(M, double, 5 * (size_t)nc); AL(fw, double, nc); AL(sa_diag, double, nc);
  AL(dWs, double, 5 * (size_t)nc); AL(dW, double, 5 * (size_t)nc); AL(dF, double, 8 * (size_t)nc);
  AL(fS, double, nf); AL(fnx, double, nf); AL(fny, double, nf); AL(fmx, double, nf); AL(fmy, double, nf);
  AL(fcx, double, nf); AL(fcy, double, nf); AL(fidL, double, nf); AL(fidR, double, nf); AL(fdn, double, nf);
  AL(lam_f, double, nf); AL(F, double, 6 * (size_t)nf); AL(sa_a, double, 4 * (size_t)nf);
  AL(G, double, 5 * (size_t)nf); AL(Gmu, double, 2 * (size_t)nf);
  AL(st, SolveState, ns); AL(dt_bits, unsigned long long, ns);
  AL(part, double, 2 * (size_t)d.n_cell_blocks); AL(err, int, 4);
  AL(hist, double, 2 * (size_t)HIST * ns);
  AL(eq40_bits, unsigned long long, ns); AL(bad, int, ns); AL(tmo, int, ns);
  d.wait_limit = ctx->opt.wait_limit > 0 ? ctx->opt.wait_limit : DEFAULT_WAIT_LIMIT;
  d.starve_test = ctx->opt.starve_test;
  d.nnz = (int)cf_face.size();
  AL(sw_cell, double, 5 * (size_t)nc); AL(sw_st, double, 4 * (size_t)d.nnz); AL(sw_j, int, d.nnz);
  UP(fs_ptr, fs_ptr); UP(fs_j, fs_j); UP(fs_slot, fs_slot); UP(cf_to_fs, cf_to_fs);
  UP(bs_ptr, bs_ptr); UP(bs_j, bs_j); UP(bs_slot, bs_slot); UP(cf_to_bs, cf_to_bs);
  d.nfs = (int)fs_j.size();
  d.nbs = (int)bs_j.size();
  AL(sc_f, double, 4 * (size_t)std::max(d.nfs, 1)); AL(sc_b, double, 4 * (size_t)std::max(d.nbs, 1));
  d.npos = P;
  UP(pos_f, pos_f); UP(pos_b, pos_b); UP(fst, fst); UP(bst, bst);
  UP(cf_to_ef, cf_to_ef); UP(cf_to_eb, cf_to_eb);
  // per-iteration records, sized for the widest sweep type
  AL(fdyn, FwdDyn<double>, (size_t)P); AL(bdyn, BwdDyn<double>, (size_t)P);
  AL(gprim, double, 6 * (size_t)nf);
  setup_sweeps();
  {
    // wide schedule: level l of every solve, solves in order
    int maxf = 0, maxb = 0;
    for (int s = 0; s < ns; s++) {
      maxf = std::max(maxf, lsp[s + 1] - lsp[s] - 1);
      maxb = std::max(maxb, blsp[s + 1] - blsp[s] - 1);
    }
    int mode = ctx->opt.sweep_mode;
    d.wide = (mode == 2) || (mode == 0 && std::max(maxf, maxb) <= WIDE_MAX_LEVELS);
    d.sweep_cluster = ctx->opt.sweep_cluster;
    std::vector<int> wf, wb;
    ctx->h_wfwd_ptr.assign(1, 0);
    ctx->h_wbwd_ptr.assign(1, 0);
    for (int l = 0; l < maxf; l++) {
      for (int s = 0; s < ns; s++)
        if (l < lsp[s + 1] - lsp[s] - 1)
          for (int k = fwd_lvl[lsp[s] + l]; k < fwd_lvl[lsp[s] + l + 1]; k++) wf.push_back(fwd_order[k]);
      ctx->h_wfwd_ptr.push_back((int)wf.size());
    }
    for (int l = 0; l < maxb; l++) {
      for (int s = 0; s < ns; s++)
        if (l < blsp[s + 1] - blsp[s] - 1)
          for (int k = bwd_lvl[blsp[s] + l]; k < bwd_lvl[blsp[s] + l + 1]; k++) wb.push_back(bwd_order[k]);
      ctx->h_wbwd_ptr.push_back((int)wb.size());
    }
    UP(wfwd_cells, wf); UP(wbwd_cells, wb);
    d.h_wfwd_ptr = ctx->h_wfwd_ptr.data();
    d.h_wbwd_ptr = ctx->h_wbwd_ptr.data();
    d.n_wfwd = maxf;
    d.n_wbwd = maxb;
  }
#undef UP
#undef AL
  CK(h2d(ctx, d.st, st.data(), sizeof(SolveState) * ns));
  std::vector<unsigned long long> inf(ns, 0x7FF0000000000000ull);
  CK(h2d(ctx, d.dt_bits, inf.data(), sizeof(unsigned long long) * ns));
  CK(cudaMallocHost((void**)&ctx->h_st, sizeof(SolveState) * ns));
  // ---- geometry, validation, wall distance ----
  launch_geometry(d, ctx->stream);
  CK(cudaGetLastError());
  int herr[4] = {0, 0, 0, 0};
  CK(cudaMemcpyAsync(herr, d.err, sizeof herr, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  if (herr[0] || herr[1]) {
    release(ctx);
    return fail(ctx, IGKS_EMESH, herr[0] ? "cell with non-positive area (cells must be CCW)"
                                         : "face normal does not point out of its left cell");
  }
  launch_wall_distance(d, ctx->stream);
  CK(cudaGetLastError());
  // free stream everywhere
  for (int s = 0; s < ns; s++) {
    std::vector<double> W(5 * (size_t)ctx->cell_pad[s], 0.0);
    for (int v = 0; v < 5; v++)
      for (int i = 0; i < ctx->meshes[s].nc; i++) W[(size_t)v * ctx->cell_pad[s] + i] = dfl[s].Winf[v];
    for (int v = 0; v < 5; v++)
      CK(h2d(ctx, d.W + (size_t)v * nc + ctx->cell_off[s], W.data() + (size_t)v * ctx->cell_pad[s],
             sizeof(double) * ctx->cell_pad[s]));
    CK(cudaStreamSynchronize(ctx->stream));
    ctx->meshes[s].nbf = 0;
  }
  for (int f : bface) ctx->meshes[fsolve[f]].nbf++;
  for (int s = 0; s < ns; s++) ctx->dev.n_solves = ns;
  CK(cudaStreamSynchronize(ctx->stream));
  ctx->built = true;
  // ---- groups of solves, one iteration of each captured as a graph ----
  rc = setup_groups(ctx);
  if (rc) { release(ctx); return rc; }
  return 0;
}

// ===================================================================================
// C ABI
// ===================================================================================

extern "C" {

int igks_create(const igks_options* opt, igks_ctx** out) {
  if (!out) return IGKS_EINVAL;
  *out = nullptr;
  igks_ctx* ctx = new igks_ctx();
  if (opt) ctx->opt = *opt;
  if (ctx->opt.check_every <= 0) ctx->opt.check_every = 20;
  if (ctx->opt.sweep_threads <= 0) ctx->opt.sweep_threads = NARROW_THREADS;
  if (ctx->opt.sweep_threads > NARROW_THREADS || ctx->opt.sweep_threads % 32) { delete ctx; return IGKS_EINVAL; }
  if (ctx->opt.wait_limit < 0 || (ctx->opt.starve_test != 0 && ctx->opt.starve_test != 1)) {
    delete ctx;
    return IGKS_EINVAL;
  }
  if (ctx->opt.precision != IGKS_PREC_FP64 && ctx->opt.precision != IGKS_PREC_MIXED &&
      ctx->opt.precision != IGKS_PREC_DF64) { delete ctx; return IGKS_EINVAL; }
  if (ctx->opt.sweep_cluster <= 0) ctx->opt.sweep_cluster = 1;
  if (ctx->opt.groups <= 0) ctx->opt.groups = 1;
  if (ctx->opt.sweep_cluster != 1 && ctx->opt.sweep_cluster != 2 && ctx->opt.sweep_cluster != 4 &&
      ctx->opt.sweep_cluster != 8) { delete ctx; return IGKS_EINVAL; }
  cudaError_t e = cudaSetDevice(ctx->opt.device);
  if (e != cudaSuccess) { delete ctx; return IGKS_ECUDA; }
  if (ctx->opt.stream) {
    ctx->stream = (cudaStream_t)ctx->opt.stream;
  } else {
    e = cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) { delete ctx; return IGKS_ECUDA; }
    ctx->own_stream = true;
  }
  *out = ctx;
  return IGKS_OK;
}

int igks_enqueue(igks_ctx* ctx, int32_t n_iters) {
  if (!ctx || n_iters < 0) return IGKS_EINVAL;
  int rc = build(ctx);
  if (rc) return rc;
  return run_iterations(ctx, n_iters);
}

int igks_kernel_times(igks_ctx* ctx, int32_t cap, float* ms, int32_t* n) {
  if (!ctx || !ms || !n || cap < 0) return IGKS_EINVAL;
  if (!ctx->opt.timing) return fail(ctx, IGKS_EBUSY, "context created without timing");
  if (!ctx->built) return fail(ctx, IGKS_EBUSY, "no iteration has run yet");
  *n = N_KERNEL_KINDS;
  for (int k = 0; k < N_KERNEL_KINDS && k < cap; k++) {
    float sum = 0.0f;
    for (int g = 0; g < ctx->n_groups; g++) {
      float t = 0.0f;
      CK(cudaEventElapsedTime(&t, ctx->gev[g][k], ctx->gev[g][k + 1]));
      sum += t;
    }
    ms[k] = sum;
  }
  return IGKS_OK;
}

const char* igks_kernel_name(int32_t i) {
  return (i >= 0 && i < N_KERNEL_KINDS) ? KERNEL_NAMES[i] : "";
}

}  // extern "C"

// host-side mesh validation shared by igks_mesh_upload and the server's submit
int igks_check_mesh_(int32_t n_nodes, const double* xy, int32_t n_cells, const int32_t* cell_ptr,
                     const int32_t* cell_nodes, int32_t n_faces, const int32_t* face_nodes,
                     const int32_t* face_cells, const int32_t* face_bc, std::string* msg) {
  auto fail = [&](int code, const char* m) { *msg = m; return code; };
  if (n_nodes <= 0 || n_cells <= 0 || n_faces <= 0 || !xy || !cell_ptr || !cell_nodes || !face_nodes ||
      !face_cells || !face_bc)
    return fail(IGKS_EINVAL, "null array or non-positive size");
  if (cell_ptr[0] != 0) return fail(IGKS_EMESH, "cell_ptr[0] != 0");
  for (int i = 0; i < n_cells; i++)
    if (cell_ptr[i + 1] - cell_ptr[i] < 3) return fail(IGKS_EMESH, "cell with fewer than 3 nodes");
  const int nk = cell_ptr[n_cells];
  for (int k = 0; k < nk; k++)
    if (cell_nodes[k] < 0 || cell_nodes[k] >= n_nodes) return fail(IGKS_EMESH, "cell node index out of range");
  std::vector<int> deg(n_cells, 0);
  for (int f = 0; f < n_faces; f++) {
    int a = face_nodes[2 * f], b = face_nodes[2 * f + 1];
    int l = face_cells[2 * f], r = face_cells[2 * f + 1];
    if (a < 0 || a >= n_nodes || b < 0 || b >= n_nodes || a == b) return fail(IGKS_EMESH, "face node index out of range");
    if (l < 0 || l >= n_cells) return fail(IGKS_EMESH, "face without a valid left cell");
    if (r >= n_cells || r == l) return fail(IGKS_EMESH, "face right cell out of range");
    if (r < 0 && (face_bc[f] < IGKS_BC_FARFIELD || face_bc[f] > IGKS_BC_MOVING_WALL))
      return fail(IGKS_EMESH, "boundary face without a boundary tag");
    if (r >= 0 && face_bc[f] != IGKS_BC_INTERIOR) return fail(IGKS_EMESH, "interior face with a boundary tag");
    deg[l]++;
    if (r >= 0) deg[r]++;
  }
  for (int i = 0; i < n_cells; i++)
    if (deg[i] != cell_ptr[i + 1] - cell_ptr[i]) return fail(IGKS_EMESH, "cell is not closed by its faces");
  // every face is an edge of its cells: a -> b in the left cell's node cycle, b -> a in the right's
  auto has_edge = [&](int c, int a, int b) {
    const int s0 = cell_ptr[c], n = cell_ptr[c + 1] - s0;
    for (int k = 0; k < n; k++)
      if (cell_nodes[s0 + k] == a && cell_nodes[s0 + (k + 1) % n] == b) return true;
    return false;
  };
  for (int f = 0; f < n_faces; f++) {
    int a = face_nodes[2 * f], b = face_nodes[2 * f + 1];
    int l = face_cells[2 * f], r = face_cells[2 * f + 1];
    if (!has_edge(l, a, b)) return fail(IGKS_EMESH, "face is not an edge of its left cell (a->b)");
    if (r >= 0 && !has_edge(r, b, a)) return fail(IGKS_EMESH, "face is not an edge of its right cell (b->a)");
  }
  for (int k = 0; k < 2 * n_nodes; k++)
    if (!std::isfinite(xy[k])) return fail(IGKS_EMESH, "non-finite node coordinate");
  return IGKS_OK;
}

bool igks_check_flow_(const igks_flow* f) {
  return f->mach > 0 && f->reynolds > 0 && f->prandtl > 0 && f->cfl_exp > 0 && f->cfl_init > 0 &&
         f->cfl_min > 0 && f->cfl_max >= f->cfl_min && f->limiter >= 0 && f->limiter <= 2 && f->t_ref > 0 &&
         f->eq40_target >= 0 && (f->scheme == IGKS_SCHEME_IMPLICIT || f->scheme == IGKS_SCHEME_EXPLICIT);
}

extern "C" {

int igks_mesh_upload(igks_ctx* ctx, int32_t n_nodes, const double* xy, int32_t n_cells,
                     const int32_t* cell_ptr, const int32_t* cell_nodes, int32_t n_faces,
                     const int32_t* face_nodes, const int32_t* face_cells, const int32_t* face_bc,
                     int32_t* solve_id) {
  if (!ctx) return IGKS_EINVAL;
  if (ctx->built) return fail(ctx, IGKS_EBUSY, "mesh upload after the device data was built");
  std::string msg;
  int vrc = igks_check_mesh_(n_nodes, xy, n_cells, cell_ptr, cell_nodes, n_faces, face_nodes, face_cells,
                             face_bc, &msg);
  if (vrc) return fail(ctx, vrc, msg);
  HostMesh m;
  m.nn = n_nodes; m.nc = n_cells; m.nf = n_faces;
  const int nk = cell_ptr[n_cells];
  m.xy.assign(xy, xy + 2 * (size_t)n_nodes);
  m.cell_ptr.assign(cell_ptr, cell_ptr + n_cells + 1);
  m.cell_nodes.assign(cell_nodes, cell_nodes + nk);
  m.face_nodes.assign(face_nodes, face_nodes + 2 * (size_t)n_faces);
  m.face_cells.assign(face_cells, face_cells + 2 * (size_t)n_faces);
  m.face_bc.assign(face_bc, face_bc + n_faces);
  ctx->meshes.push_back(std::move(m));
  ctx->flows.push_back(default_flow());
  ctx->flow_set.push_back(0);
  if (solve_id) *solve_id = (int32_t)ctx->meshes.size() - 1;
  return IGKS_OK;
}

int igks_set_flow(igks_ctx* ctx, int32_t solve, const igks_flow* f) {
  if (!ctx || !f || solve < 0 || solve >= (int)ctx->meshes.size()) return IGKS_EINVAL;
  if (!igks_check_flow_(f)) return fail(ctx, IGKS_EINVAL, "invalid flow conditions");
  ctx->flows[solve] = *f;
  ctx->flow_set[solve] = 1;
  if (ctx->built) {
    DevFlow d = make_devflow(*f);
    CK(h2d(ctx, (DevFlow*)ctx->dev.flow + solve, &d, sizeof d));
    CK(cudaStreamSynchronize(ctx->stream));
  }
  return IGKS_OK;
}

static int check_solve(igks_ctx* ctx, int32_t solve) {
  if (!ctx || solve < 0 || solve >= (int)ctx->meshes.size()) return IGKS_EINVAL;
  return 0;
}

int igks_init_freestream(igks_ctx* ctx, int32_t solve) {
  if (check_solve(ctx, solve)) return IGKS_EINVAL;
  int rc = build(ctx);
  if (rc) return rc;
  const HostMesh& m = ctx->meshes[solve];
  DevFlow fl = make_devflow(ctx->flows[solve]);
  std::vector<double> W((size_t)m.nc);
  for (int v = 0; v < 5; v++) {
    std::fill(W.begin(), W.end(), fl.Winf[v]);
    CK(h2d(ctx, ctx->dev.W + (size_t)v * ctx->nc_pad + ctx->cell_off[solve], W.data(), sizeof(double) * m.nc));
    CK(cudaStreamSynchronize(ctx->stream));
  }
  double sc[5] = {0.0, ctx->flows[solve].cfl_init, 0.0, 0.0, 0.0};
  return igks_set_scalars(ctx, solve, sc);
}

int igks_iterate(igks_ctx* ctx, int32_t max_iters, igks_status* status) {
  if (!ctx || max_iters < 0) return IGKS_EINVAL;
  int rc = build(ctx);
  if (rc) return rc;
  CK(cudaSetDevice(ctx->opt.device));
  const int ns = ctx->dev.n_solves;
  int done = 0;
  bool any_live = true;
  while (done < max_iters && any_live) {
    int k = std::min(ctx->opt.check_every, max_iters - done);
    rc = run_iterations(ctx, k);
    if (rc) return rc;
    done += k;
    CK(cudaMemcpyAsync(ctx->h_st, ctx->dev.st, sizeof(SolveState) * ns, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    any_live = false;
    for (int s = 0; s < ns; s++) any_live |= (ctx->h_st[s].state == 0);
  }
  if (max_iters == 0) {
    CK(cudaMemcpyAsync(ctx->h_st, ctx->dev.st, sizeof(SolveState) * ns, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
  }
  bool all_conv = true, any_div = false;
  for (int s = 0; s < ns; s++) {
    const SolveState& q = ctx->h_st[s];
    if (status) {
      igks_status& o = status[s];
      o.iters = q.iter; o.state = q.state; o.res_l2_rho = q.res_l2;
      o.res_l2_rel = q.res_l2_first > 0 ? q.res_l2 / q.res_l2_first : 0.0;
      o.res_inf = q.res_inf; o.eq40_ratio = q.eq40; o.cfl = q.cfl; o.dt = q.dt;
    }
    all_conv &= (q.state == IGKS_CONVERGED);
    any_div |= (q.state < 0);
  }
  for (int s = 0; s < ns; s++)
    if (ctx->h_st[s].state == IGKS_TIMEOUT) return fail(ctx, IGKS_TIMEOUT, "a sweep wait ran out of its spin limit");
  if (any_div) return IGKS_DIVERGED;
  return all_conv ? IGKS_CONVERGED : IGKS_OK;
}

// copy k components of a per-cell [k][nc_pad] array of a solve into out[k][n]
static int get_cells(igks_ctx* ctx, int solve, const double* base, int k, double* out) {
  const int n = ctx->meshes[solve].nc;
  CK(d2h_2d(ctx, out, sizeof(double) * n, base + ctx->cell_off[solve], sizeof(double) * ctx->nc_pad,
            sizeof(double) * n, k));
  return 0;
}

static int get_faces(igks_ctx* ctx, int solve, const double* base, int k, double* out) {
  const int n = ctx->meshes[solve].nf;
  CK(d2h_2d(ctx, out, sizeof(double) * n, base + ctx->face_off[solve], sizeof(double) * ctx->nf,
            sizeof(double) * n, k));
  return 0;
}

int igks_get_fields(igks_ctx* ctx, int32_t solve, double* W) {
  if (check_solve(ctx, solve) || !W) return IGKS_EINVAL;
  int rc = build(ctx);
  if (rc) return rc;
  CK(cudaStreamSynchronize(ctx->stream));
  return get_cells(ctx, solve, ctx->dev.W, 5, W);
}

int igks_set_fields(igks_ctx* ctx, int32_t solve, const double* W) {
  if (check_solve(ctx, solve) || !W) return IGKS_EINVAL;
  int rc = build(ctx);
  if (rc) return rc;
  const int n = ctx->meshes[solve].nc;
  for (int i = 0; i < n; i++)
    if (!(W[i] > 0.0) || !std::isfinite(W[3 * (size_t)n + i])) return fail(ctx, IGKS_EINVAL, "non-physical state");
  CK(cudaStreamSynchronize(ctx->stream));
  CK(h2d_2d(ctx, ctx->dev.W + ctx->cell_off[solve], sizeof(double) * ctx->nc_pad, W, sizeof(double) * n,
            sizeof(double) * n, 5));
  CK(cudaStreamSynchronize(ctx->stream));
  return IGKS_OK;
}

int igks_get_fields_all(igks_ctx* ctx, double* W) {
  if (!ctx || !W || ctx->meshes.empty()) return IGKS_EINVAL;
  int rc = build(ctx);
  if (rc) return rc;
  size_t N = 0;
  for (const HostMesh& m : ctx->meshes) N += m.nc;
  size_t off = 0;
  for (size_t k = 0; k < ctx->meshes.size(); k++) {
    const size_t n = ctx->meshes[k].nc;
    CK(cudaMemcpy2DAsync(W + off, sizeof(double) * N, ctx->dev.W + ctx->cell_off[k], sizeof(double) * ctx->nc_pad,
                         sizeof(double) * n, 5, cudaMemcpyDeviceToHost, ctx->stream));
    off += n;
  }
  CK(cudaStreamSynchronize(ctx->stream));
  return IGKS_OK;
}

int igks_set_fields_all(igks_ctx* ctx, const double* W) {
  if (!ctx || !W || ctx->meshes.empty()) return IGKS_EINVAL;
  int rc = build(ctx);
  if (rc) return rc;
  Dev& d = ctx->dev;
  const int ns = d.n_solves;
  size_t N = 0;
  for (const HostMesh& m : ctx->meshes) N += m.nc;
  double* staged = (double*)d.dW;                  // [5][nc_pad] doubles, scratch between iterations
  size_t off = 0;
  for (size_t k = 0; k < ctx->meshes.size(); k++) {
    const size_t n = ctx->meshes[k].nc;
    CK(cudaMemcpy2DAsync(staged + ctx->cell_off[k], sizeof(double) * ctx->nc_pad, W + off, sizeof(double) * N,
                         sizeof(double) * n, 5, cudaMemcpyHostToDevice, ctx->stream));
    off += n;
  }
  CK(cudaMemsetAsync(d.bad, 0, sizeof(int) * ns, ctx->stream));
  launch_set_state(d, staged, d.bad, ctx->stream);
  CK(cudaGetLastError());
  std::vector<int> bad(ns, 0);
  CK(cudaMemcpyAsync(bad.data(), d.bad, sizeof(int) * ns, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaMemsetAsync(d.bad, 0, sizeof(int) * ns, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  for (int s = 0; s < ns; s++)
    if (bad[s]) return fail(ctx, IGKS_EINVAL, "non-physical state (solve " + std::to_string(s) + " kept its state)");
  return IGKS_OK;
}

int igks_get_scalars(igks_ctx* ctx, int32_t solve, double* out) {
  if (check_solve(ctx, solve) || !out) return IGKS_EINVAL;
  int rc = build(ctx);
  if (rc) return rc;
  SolveState q;
  CK(cudaStreamSynchronize(ctx->stream));
  CK(d2h(ctx, &q, ctx->dev.st + solve, sizeof q));
  out[0] = q.iter; out[1] = q.cfl; out[2] = q.res_inf_prev; out[3] = q.res_l2_first; out[4] = q.state;
  return IGKS_OK;
}

int igks_set_scalars(igks_ctx* ctx, int32_t solve, const double* in) {
  if (check_solve(ctx, solve) || !in) return IGKS_EINVAL;
  int rc = build(ctx);
  if (rc) return rc;
  SolveState q;
  CK(cudaStreamSynchronize(ctx->stream));
  CK(d2h(ctx, &q, ctx->dev.st + solve, sizeof q));
  q.iter = (int)in[0]; q.cfl = in[1]; q.res_inf_prev = in[2]; q.res_l2_first = in[3]; q.state = (int)in[4];
  q.pending = 0;
  CK(h2d(ctx, ctx->dev.st + solve, &q, sizeof q));
  CK(cudaStreamSynchronize(ctx->stream));
  return IGKS_OK;
}

int igks_get_array(igks_ctx* ctx, int32_t solve, int32_t which, double* out) {
  if (check_solve(ctx, solve) || !out) return IGKS_EINVAL;
  int rc = build(ctx);
  if (rc) return rc;
  CK(cudaStreamSynchronize(ctx->stream));
  const Dev& d = ctx->dev;
  const int n = ctx->meshes[solve].nc, nf = ctx->meshes[solve].nf;
  switch (which) {
    case IGKS_ARR_GRAD: return get_cells(ctx, solve, d.grad, 8, out);
    case IGKS_ARR_PHI: return get_cells(ctx, solve, d.phi, 4, out);
    case IGKS_ARR_LAMBDA_F: return get_faces(ctx, solve, d.lam_f, 1, out);
    case IGKS_ARR_LAMBDA_C: return get_cells(ctx, solve, d.Lam, 1, out);
    case IGKS_ARR_FLUX: return get_faces(ctx, solve, d.F, 6, out);
    case IGKS_ARR_RES: return get_cells(ctx, solve, d.M, 5, out);
    case IGKS_ARR_GHOST: {
      rc = get_faces(ctx, solve, d.G, 5, out);
      if (rc) return rc;
      for (int f = 0; f < nf; f++)
        if (ctx->meshes[solve].face_cells[2 * f + 1] >= 0)
          for (int v = 0; v < 5; v++) out[(size_t)v * nf + f] = 0.0;
      return 0;
    }
    case IGKS_ARR_DWSTAR:
    case IGKS_ARR_DW: {
      const void* src = which == IGKS_ARR_DWSTAR ? d.dWs : d.dW;
      if (ctx->opt.precision == IGKS_PREC_MIXED) {
        std::vector<float> tmp(5 * (size_t)n);
        CK(d2h_2d(ctx, tmp.data(), sizeof(float) * n, (const float*)src + ctx->cell_off[solve],
                  sizeof(float) * ctx->nc_pad, sizeof(float) * n, 5));
        for (size_t k = 0; k < tmp.size(); k++) out[k] = tmp[k];
        return 0;
      }
      if (ctx->opt.precision == IGKS_PREC_DF64) {   // pairs (hi, lo) of floats
        std::vector<float> tmp(10 * (size_t)n);
        CK(d2h_2d(ctx, tmp.data(), 2 * sizeof(float) * n, (const float*)src + 2 * (size_t)ctx->cell_off[solve],
                  2 * sizeof(float) * ctx->nc_pad, 2 * sizeof(float) * n, 5));
        for (size_t k = 0; k < 5 * (size_t)n; k++) out[k] = (double)tmp[2 * k] + (double)tmp[2 * k + 1];
        return 0;
      }
      return get_cells(ctx, solve, (const double*)src, 5, out);
    }
    case IGKS_ARR_GEOM_CELL:
      if ((rc = get_cells(ctx, solve, d.area, 1, out))) return rc;
      if ((rc = get_cells(ctx, solve, d.cx, 1, out + n))) return rc;
      if ((rc = get_cells(ctx, solve, d.cy, 1, out + 2 * (size_t)n))) return rc;
      return get_cells(ctx, solve, d.wall_d, 1, out + 3 * (size_t)n);
    case IGKS_ARR_GEOM_FACE:
      if ((rc = get_faces(ctx, solve, d.fS, 1, out))) return rc;
      if ((rc = get_faces(ctx, solve, d.fnx, 1, out + nf))) return rc;
      if ((rc = get_faces(ctx, solve, d.fny, 1, out + 2 * (size_t)nf))) return rc;
      if ((rc = get_faces(ctx, solve, d.fmx, 1, out + 3 * (size_t)nf))) return rc;
      return get_faces(ctx, solve, d.fmy, 1, out + 4 * (size_t)nf);
  }
  return fail(ctx, IGKS_EINVAL, "unknown array id");
}

int igks_get_history(igks_ctx* ctx, int32_t solve, int32_t cap, double* out, int32_t* n) {
  if (check_solve(ctx, solve) || !n || cap < 0 || (cap > 0 && !out)) return IGKS_EINVAL;
  int rc = build(ctx);
  if (rc) return rc;
  SolveState q;
  CK(cudaStreamSynchronize(ctx->stream));
  CK(d2h(ctx, &q, ctx->dev.st + solve, sizeof q));
  std::vector<double> h(2 * (size_t)HIST);
  CK(d2h(ctx, h.data(), ctx->dev.hist + (size_t)solve * HIST * 2, sizeof(double) * h.size()));
  const int m = std::min({q.iter, HIST, (int)cap});
  for (int k = 0; k < m; k++) {
    const int it = q.iter - m + k;            // 0-based iteration index
    out[3 * k] = it + 1;
    out[3 * k + 1] = h[2 * (it % HIST)];
    out[3 * k + 2] = h[2 * (it % HIST) + 1];
  }
  *n = m;
  return IGKS_OK;
}

int igks_mesh_info(igks_ctx* ctx, int32_t solve, int32_t* out) {
  if (check_solve(ctx, solve) || !out) return IGKS_EINVAL;
  int rc = build(ctx);
  if (rc) return rc;
  const HostMesh& m = ctx->meshes[solve];
  out[0] = m.nc; out[1] = m.nf; out[2] = m.nlev_f; out[3] = m.nlev_b; out[4] = m.nbf;
  return IGKS_OK;
}

int igks_get_forces(igks_ctx* ctx, int32_t solve, int32_t bc_tag, double* out) {
  if (check_solve(ctx, solve) || !out) return IGKS_EINVAL;
  int rc = build(ctx);
  if (rc) return rc;
  const HostMesh& m = ctx->meshes[solve];
  std::vector<double> F(6 * (size_t)m.nf), G(5 * (size_t)m.nf), geo(5 * (size_t)m.nf);
  SolveState q;
  CK(cudaStreamSynchronize(ctx->stream));
  CK(d2h(ctx, &q, ctx->dev.st + solve, sizeof q));
  if ((rc = get_faces(ctx, solve, ctx->dev.F, 6, F.data()))) return rc;
  if ((rc = get_faces(ctx, solve, ctx->dev.G, 5, G.data()))) return rc;
  if ((rc = igks_get_array(ctx, solve, IGKS_ARR_GEOM_FACE, geo.data()))) return rc;
  if (!(q.dt > 0.0)) return fail(ctx, IGKS_EBUSY, "no iteration has run yet");
  double fx = 0, fy = 0, vx = 0, vy = 0;
  const int nf = m.nf;
  for (int f = 0; f < nf; f++) {
    if (m.face_cells[2 * f + 1] >= 0 || m.face_bc[f] != bc_tag) continue;
    // momentum through the face per unit time = force of the fluid on the boundary
    double px = F[(size_t)nf + f] / q.dt, py = F[2 * (size_t)nf + f] / q.dt;
    fx += px; fy += py;
    double r = G[f], mx = G[(size_t)nf + f], my = G[2 * (size_t)nf + f], E = G[3 * (size_t)nf + f];
    double p = (GAMMA - 1.0) * (E - 0.5 * (mx * mx + my * my) / r);
    double S = geo[f], nx = geo[(size_t)nf + f], ny = geo[2 * (size_t)nf + f];
    vx += px - p * nx * S;
    vy += py - p * ny * S;
  }
  double a = ctx->flows[solve].aoa_deg * M_PI / 180.0;
  double ca = std::cos(a), sa = std::sin(a);
  out[0] = 2.0 * (-fx * sa + fy * ca);
  out[1] = 2.0 * (fx * ca + fy * sa);
  out[2] = 2.0 * (vx * ca + vy * sa);
  return IGKS_OK;
}

int igks_order_cells(int32_t n_cells, int32_t n_faces, const int32_t* face_cells, int32_t mode, int32_t* perm,
                     int32_t* n_colors) {
  if (n_cells <= 0 || n_faces < 0 || !face_cells || !perm || (mode != 0 && mode != 1)) return IGKS_EINVAL;
  if (mode == 0) {
    for (int i = 0; i < n_cells; i++) perm[i] = i;
    if (n_colors) *n_colors = 1;
    return IGKS_OK;
  }
  // adjacency through interior faces
  std::vector<int> ptr(n_cells + 1, 0), adj;
  for (int f = 0; f < n_faces; f++) {
    int l = face_cells[2 * f], r = face_cells[2 * f + 1];
    if (l < 0 || l >= n_cells || r >= n_cells) return IGKS_EMESH;
    if (r >= 0) { ptr[l + 1]++; ptr[r + 1]++; }
  }
  for (int i = 0; i < n_cells; i++) ptr[i + 1] += ptr[i];
  adj.assign(ptr[n_cells], 0);
  {
    std::vector<int> fill(ptr.begin(), ptr.end() - 1);
    for (int f = 0; f < n_faces; f++) {
      int l = face_cells[2 * f], r = face_cells[2 * f + 1];
      if (r >= 0) { adj[fill[l]++] = r; adj[fill[r]++] = l; }
    }
  }
  // greedy colouring in index order: smallest colour not used by a coloured neighbour
  std::vector<int> col(n_cells, -1), mark;
  int nc = 0;
  for (int i = 0; i < n_cells; i++) {
    mark.assign(nc + 1, 0);
    for (int k = ptr[i]; k < ptr[i + 1]; k++)
      if (col[adj[k]] >= 0) mark[col[adj[k]]] = 1;
    int c = 0;
    while (c < nc && mark[c]) c++;
    col[i] = c;
    nc = std::max(nc, c + 1);
  }
  // stable order by colour
  std::vector<int> cnt(nc + 1, 0);
  for (int i = 0; i < n_cells; i++) cnt[col[i] + 1]++;
  for (int c = 0; c < nc; c++) cnt[c + 1] += cnt[c];
  for (int i = 0; i < n_cells; i++) perm[cnt[col[i]]++] = i;
  if (n_colors) *n_colors = nc;
  return IGKS_OK;
}

// re-capture the iteration graphs after a launch parameter changed
static int recapture(igks_ctx* ctx) { return setup_groups(ctx); }

int igks_autotune(igks_ctx* ctx, int32_t iters_per_trial, igks_tuning* out) {
  if (!ctx || iters_per_trial <= 0) return IGKS_EINVAL;
  int rc = build(ctx);
  if (rc) return rc;
  Dev& d = ctx->dev;
  const int ns = d.n_solves;
  // the state every trial starts from (per-cell fields and per-solve iteration state)
  double* Wb = nullptr;
  SolveState* Sb = nullptr;
  unsigned long long* Tb = nullptr;
  const size_t wbytes = sizeof(double) * 5 * (size_t)ctx->nc_pad;
  CK(cudaMalloc(&Wb, wbytes));
  CK(cudaMalloc(&Sb, sizeof(SolveState) * ns));
  CK(cudaMalloc(&Tb, sizeof(unsigned long long) * ns));
  auto save = [&]() {
    cudaMemcpyAsync(Wb, d.W, wbytes, cudaMemcpyDeviceToDevice, ctx->stream);
    cudaMemcpyAsync(Sb, d.st, sizeof(SolveState) * ns, cudaMemcpyDeviceToDevice, ctx->stream);
    cudaMemcpyAsync(Tb, d.dt_bits, sizeof(unsigned long long) * ns, cudaMemcpyDeviceToDevice, ctx->stream);
  };
  auto restore = [&]() {
    cudaMemcpyAsync(d.W, Wb, wbytes, cudaMemcpyDeviceToDevice, ctx->stream);
    cudaMemcpyAsync(d.st, Sb, sizeof(SolveState) * ns, cudaMemcpyDeviceToDevice, ctx->stream);
    cudaMemcpyAsync(d.dt_bits, Tb, sizeof(unsigned long long) * ns, cudaMemcpyDeviceToDevice, ctx->stream);
    cudaMemsetAsync(d.eq40_bits, 0, sizeof(unsigned long long) * ns, ctx->stream);
    cudaMemsetAsync(d.bad, 0, sizeof(int) * ns, ctx->stream);
  };
  save();
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  igks_tuning best{};
  best.ms_per_iter = 1e30f;
  const bool wide_ok = std::max(d.n_wfwd, d.n_wbwd) <= 4 * WIDE_MAX_LEVELS;
  const int flux_blocks[] = {64, 128};
  const int sweep_threads[] = {128, 256};
  const int clusters[] = {1, 2, 4};
  const int groups[] = {1, 2, 4, 8};
  int err = 0;
  for (int wide = 0; wide <= (wide_ok ? 1 : 0) && !err; wide++)
    for (int fb : flux_blocks)
      for (int stt : sweep_threads)
        for (int cl : clusters)
          for (int gr : groups) {
          if (wide && (stt != sweep_threads[0] || cl != 1 || gr != 1)) continue;   // the wide schedule has its own block
          if (gr > 1 && (cl != 1 || gr > ns)) continue;
          d.wide = wide;
          d.flux_block = fb;
          d.sweep_cluster = cl;
          ctx->opt.sweep_threads = stt;
          ctx->opt.groups = gr;
          if ((err = recapture(ctx))) break;
          restore();
          if ((err = run_iterations(ctx, 1))) break;     // the first iteration warms up
          cudaEventRecord(e0, ctx->stream);
          if ((err = run_iterations(ctx, iters_per_trial))) break;
          cudaEventRecord(e1, ctx->stream);
          if (cudaEventSynchronize(e1) != cudaSuccess) { err = IGKS_ECUDA; break; }
          float ms = 0.0f;
          cudaEventElapsedTime(&ms, e0, e1);
          ms /= iters_per_trial;
          if (ms < best.ms_per_iter) best = igks_tuning{stt, fb, wide ? 2 : 1, cl, ms, gr};
          }
  // apply the winner and put every solve back where it was
  d.wide = best.sweep_mode == 2;
  d.flux_block = best.flux_block;
  d.sweep_cluster = best.sweep_cluster;
  ctx->opt.sweep_threads = best.sweep_threads;
  ctx->opt.sweep_mode = best.sweep_mode;
  ctx->opt.sweep_cluster = best.sweep_cluster;
  ctx->opt.groups = best.groups;
  if (!err) err = recapture(ctx);
  restore();
  cudaStreamSynchronize(ctx->stream);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(Wb);
  cudaFree(Sb);
  cudaFree(Tb);
  CK(cudaGetLastError());
  if (err) return fail(ctx, err, "autotune trial failed");
  if (out) *out = best;
  return IGKS_OK;
}

int igks_set_launch(igks_ctx* ctx, const igks_tuning* t) {
  if (!ctx || !t) return IGKS_EINVAL;
  if ((t->sweep_threads != 128 && t->sweep_threads != 256) || (t->flux_block != 64 && t->flux_block != 128) ||
      (t->sweep_mode != 1 && t->sweep_mode != 2) ||
      (t->sweep_cluster != 1 && t->sweep_cluster != 2 && t->sweep_cluster != 4 && t->sweep_cluster != 8) ||
      t->groups < 1)
    return fail(ctx, IGKS_EINVAL, "launch configuration outside the tuner's choices");
  int rc = build(ctx);
  if (rc) return rc;
  Dev& d = ctx->dev;
  d.wide = t->sweep_mode == 2;
  d.flux_block = t->flux_block;
  d.sweep_cluster = t->sweep_cluster;
  ctx->opt.sweep_threads = t->sweep_threads;
  ctx->opt.sweep_mode = t->sweep_mode;
  ctx->opt.sweep_cluster = t->sweep_cluster;
  ctx->opt.groups = t->groups;
  return recapture(ctx);
}

int igks_launches_per_iteration(igks_ctx* ctx, int32_t* out) {
  if (!ctx || !out) return IGKS_EINVAL;
  int rc = build(ctx);
  if (rc) return rc;
  *out = ctx->n_groups * (N_KERNEL_KINDS - 2 + (ctx->dev.wide ? ctx->dev.n_wfwd + ctx->dev.n_wbwd : 2));
  return IGKS_OK;
}

int igks_destroy(igks_ctx* ctx) {
  if (!ctx) return IGKS_EINVAL;
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  release(ctx);
  if (ctx->own_stream && ctx->stream) cudaStreamDestroy(ctx->stream);
  delete ctx;
  return IGKS_OK;
}

int igks_footprint_bytes(int32_t n_nodes, int32_t n_cells, int32_t n_faces, int32_t nnz, int64_t* out) {
  if (n_nodes <= 0 || n_cells <= 0 || n_faces <= 0 || nnz < 0 || !out) return IGKS_EINVAL;
  const int64_t ncp = (int64_t)(n_cells + CELL_ALIGN - 1) / CELL_ALIGN * CELL_ALIGN;
  // (plus 16 KiB of residual history per solve, in the fixed part below)
  // per padded cell: 62 doubles (state, gradients, speeds, increments, cell constants),
  // the sweep records (2 x 48 B static, 2 x 272 B per iteration), 9 ints (CSR pointers,
  // orders, levels, positions) and 16 B to spare; per CSR entry 60 B (face and node lists, sweep
  // stencil coefficients, maps) + 40 B (one sweep entry); per face 34 doubles + 8 ints; per
  // node 2 doubles; a few hundred bytes per solve
  *out = 1188 * ncp + 100 * (int64_t)nnz + 304 * (int64_t)n_faces + 16 * (int64_t)n_nodes + 4096 + 16384;
  return IGKS_OK;
}

int igks_device_bytes(igks_ctx* ctx, int64_t* out) {
  if (!ctx || !out) return IGKS_EINVAL;
  int64_t b = 0;
  for (const auto& x : ctx->bufs) b += (int64_t)x.bytes;
  *out = b;
  return IGKS_OK;
}

const char* igks_last_error(igks_ctx* ctx) {
  if (!ctx) return igks_noalloc_last_error_();
  return ctx->err.c_str();
}

}  // extern "C"
