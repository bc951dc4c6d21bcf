// igks_server.cu -- continuous batching of steady solves (host code over the context
// API of igks_api.cu; no kernels of its own).
//
// Requests wait in a FIFO queue. Each step admits the queue head into one new cohort (a
// context on its own stream) while slots and the HBM budget allow, moves the live solves
// of sparse cohorts into it, runs a fixed number of iterations on every cohort with the
// cohorts' graphs in flight together, and retires what stopped. A solve's arithmetic does
// not depend on its cohort (each kernel works per solve; converged solves are skipped on
// the device), and a move copies its fields and iteration state exactly, so its result is
// bitwise that of a context of its own.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <deque>
#include <map>
#include <string>
#include <vector>

#include "../../include/igks.h"

// igks_api.cu
int igks_check_mesh_(int32_t n_nodes, const double* xy, int32_t n_cells, const int32_t* cell_ptr,
                     const int32_t* cell_nodes, int32_t n_faces, const int32_t* face_nodes,
                     const int32_t* face_cells, const int32_t* face_bc, std::string* msg);
bool igks_check_flow_(const igks_flow* f);

namespace {

struct Request {
  int64_t id = 0, tag = 0;
  int32_t nn = 0, nc = 0, nf = 0;
  std::vector<double> xy;
  std::vector<int32_t> cell_ptr, cell_nodes, face_nodes, face_cells, face_bc;
  igks_flow flow{};
  double t_submit = 0.0, t_admit = 0.0;
  int64_t footprint = 0;
  // state of a live solve moved out of a cohort that is being freed
  bool carried = false;
  std::vector<double> W;
  std::vector<double> W0;   // the request's starting state (empty: free stream)
  double scal[5] = {0, 0, 0, 0, 0};
};

struct Member {
  Request req;
  int32_t sid = 0;
  bool live = true;
};

struct Cohort {
  igks_ctx* ctx = nullptr;
  int32_t serial = 0;
  std::vector<Member> members;
  int64_t bytes = 0;    // summed footprints of its solves
  int64_t cells = 0;
};

}  // namespace

struct igks_server {
  igks_server_options opt{};
  std::chrono::steady_clock::time_point t0;
  std::deque<Request> queue;
  std::vector<Cohort> cohorts;
  std::deque<igks_result> done;
  std::map<int64_t, std::vector<double>> fields;
  int64_t next_id = 0;
  int32_t next_cohort = 0;
  int32_t last_admitted = 0, last_repacked = 0;
  double last_step = 0.0;
  std::string err;
};

static double now_s(const igks_server* s) {
  return std::chrono::duration<double>(std::chrono::steady_clock::now() - s->t0).count();
}

static int sfail(igks_server* s, int code, const std::string& msg) {
  s->err = msg;
  return code;
}

static int ctx_fail(igks_server* s, igks_ctx* ctx, int code, const char* what) {
  return sfail(s, code, std::string(what) + ": " + igks_last_error(ctx));
}

static int64_t live_cells(const Cohort& c) {
  int64_t n = 0;
  for (const Member& m : c.members)
    if (m.live) n += m.req.nc;
  return n;
}

static int n_live(const igks_server* s) {
  int n = 0;
  for (const Cohort& c : s->cohorts)
    for (const Member& m : c.members) n += m.live;
  return n;
}

static int64_t resident_bytes(const igks_server* s) {
  int64_t b = 0;
  for (const Cohort& c : s->cohorts) b += c.bytes;
  return b;
}

// copy a live member's fields and iteration state to the host
static int carry_out(igks_server* s, Cohort& c, Member& m) {
  m.req.W.resize(5 * (size_t)m.req.nc);
  int rc = igks_get_fields(c.ctx, m.sid, m.req.W.data());
  if (rc) return ctx_fail(s, c.ctx, rc, "moving a live solve");
  rc = igks_get_scalars(c.ctx, m.sid, m.req.scal);
  if (rc) return ctx_fail(s, c.ctx, rc, "moving a live solve");
  m.req.carried = true;
  return 0;
}

// build one cohort context from requests (moved solves resume their state)
static int build_cohort(igks_server* s, std::vector<Request>& reqs, Cohort& out) {
  igks_options o{};
  o.precision = s->opt.precision;
  o.device = s->opt.device;
  o.use_graph = 1;
  o.check_every = 1 << 20;
  igks_ctx* ctx = nullptr;
  int rc = igks_create(&o, &ctx);
  if (rc) return sfail(s, rc, "igks_create failed for a cohort");
  out = Cohort{};
  out.ctx = ctx;
  std::vector<int32_t> sids;
  for (Request& r : reqs) {
    int32_t sid = -1;
    rc = igks_mesh_upload(ctx, r.nn, r.xy.data(), r.nc, r.cell_ptr.data(), r.cell_nodes.data(), r.nf,
                          r.face_nodes.data(), r.face_cells.data(), r.face_bc.data(), &sid);
    if (!rc) rc = igks_set_flow(ctx, sid, &r.flow);
    if (rc) {
      int code = ctx_fail(s, ctx, rc, "cohort upload");
      igks_destroy(ctx);
      out.ctx = nullptr;
      return code;
    }
    sids.push_back(sid);
  }
  for (size_t k = 0; k < reqs.size(); k++) {
    out.bytes += reqs[k].footprint;
    out.cells += reqs[k].nc;
    out.members.push_back(Member{std::move(reqs[k]), sids[k], true});
  }
  reqs.clear();
  for (Member& m : out.members) {
    if (m.req.carried) {
      rc = igks_set_fields(ctx, m.sid, m.req.W.data());
      if (!rc) rc = igks_set_scalars(ctx, m.sid, m.req.scal);
    } else {
      rc = igks_init_freestream(ctx, m.sid);
      if (!rc && !m.req.W0.empty()) rc = igks_set_fields(ctx, m.sid, m.req.W0.data());
    }
    if (rc) break;
  }
  if (rc) {
    int code = ctx_fail(s, ctx, rc, "cohort start");
    // hand the requests back so that nothing is lost
    for (Member& m : out.members) reqs.push_back(std::move(m.req));
    igks_destroy(ctx);
    out = Cohort{};
    return code;
  }
  for (Member& m : out.members) {
    m.req.carried = false;
    m.req.W.clear();
    m.req.W.shrink_to_fit();
    m.req.W0.clear();
    m.req.W0.shrink_to_fit();
  }
  out.serial = s->next_cohort++;
  return 0;
}

static int admit(igks_server* s) {
  const int64_t budget = s->opt.hbm_budget;
  const int live = n_live(s);
  // sparse cohorts: live cells below repack_fraction of their cells
  std::vector<size_t> sparse;
  int64_t freed = 0;
  if (s->opt.repack_fraction > 0.0)
    for (size_t k = 0; k < s->cohorts.size(); k++) {
      const Cohort& c = s->cohorts[k];
      const int64_t lc = live_cells(c);
      if (lc > 0 && (double)lc < s->opt.repack_fraction * (double)c.cells) {
        sparse.push_back(k);
        int64_t live_fp = 0;
        for (const Member& m : c.members)
          if (m.live) live_fp += m.req.footprint;
        freed += c.bytes - live_fp;
      }
    }
  const int64_t bytes_if_repacked = resident_bytes(s) - freed;
  // queue head, in order, while a slot is free and the budget holds it
  size_t take = 0;
  int64_t take_bytes = 0;
  while (take < s->queue.size() && (int)take < s->opt.max_cohort && live + (int)take < s->opt.max_slots) {
    const Request& r = s->queue[take];
    if (bytes_if_repacked + take_bytes + r.footprint > budget) break;
    take_bytes += r.footprint;
    take++;
  }
  const bool repack = !sparse.empty() && (take > 0 || sparse.size() >= 2);
  if (take == 0 && !repack) return 0;
  std::vector<Request> reqs;
  int moved = 0;
  if (repack) {
    // copy the live solves out, then free their cohorts before the new one is built
    for (size_t k : sparse) {
      Cohort& c = s->cohorts[k];
      for (Member& m : c.members)
        if (m.live) {
          int rc = carry_out(s, c, m);
          if (rc) return rc;
          reqs.push_back(std::move(m.req));
          moved++;
        }
      igks_destroy(c.ctx);
      c.ctx = nullptr;
    }
    std::vector<Cohort> keep;
    for (Cohort& c : s->cohorts)
      if (c.ctx) keep.push_back(std::move(c));
    s->cohorts.swap(keep);
  }
  const double t = now_s(s);
  for (size_t k = 0; k < take; k++) {
    Request r = std::move(s->queue.front());
    s->queue.pop_front();
    r.t_admit = t;
    reqs.push_back(std::move(r));
  }
  Cohort c;
  int rc = build_cohort(s, reqs, c);
  if (rc) {
    // back to the queue head in their order (moved solves keep their carried state)
    for (auto it = reqs.rbegin(); it != reqs.rend(); ++it) s->queue.push_front(std::move(*it));
    return rc;
  }
  s->cohorts.push_back(std::move(c));
  s->last_admitted = (int)take;
  s->last_repacked = moved;
  return 0;
}

static int run(igks_server* s) {
  for (Cohort& c : s->cohorts) {
    if (live_cells(c) == 0) continue;
    int rc = igks_enqueue(c.ctx, s->opt.iters_per_step);
    if (rc) return ctx_fail(s, c.ctx, rc, "enqueue");
  }
  return 0;
}

static int retire(igks_server* s) {
  std::vector<igks_status> st;
  for (Cohort& c : s->cohorts) {
    st.assign(c.members.size(), igks_status{});
    int rc = igks_iterate(c.ctx, 0, st.data());   // waits for the cohort's stream
    if (rc < 0 && rc != IGKS_DIVERGED) return ctx_fail(s, c.ctx, rc, "reading solve states");
    for (Member& m : c.members) {
      if (!m.live) continue;
      const igks_status& q = st[m.sid];
      if (q.state == 0 && q.iters < s->opt.max_iters) continue;
      igks_result r{};
      r.id = m.req.id;
      r.tag = m.req.tag;
      r.state = q.state == 0 ? IGKS_MAXITER : q.state;
      r.iters = q.iters;
      r.n_cells = m.req.nc;
      r.cohort = c.serial;
      r.res_l2_rel = q.res_l2_rel;
      r.t_submit = m.req.t_submit;
      r.t_admit = m.req.t_admit;
      r.footprint = m.req.footprint;
      if (q.state == 0) {
        // stop it on the device: every kernel skips a solve whose state is not 0
        double sc[5];
        rc = igks_get_scalars(c.ctx, m.sid, sc);
        if (!rc) { sc[4] = IGKS_MAXITER; rc = igks_set_scalars(c.ctx, m.sid, sc); }
        if (rc) return ctx_fail(s, c.ctx, rc, "stopping a solve at the iteration cap");
      }
      if (igks_get_forces(c.ctx, m.sid, IGKS_BC_WALL, r.forces) != IGKS_OK)
        r.forces[0] = r.forces[1] = r.forces[2] = NAN;
      if (s->opt.keep_fields) {
        std::vector<double> W(5 * (size_t)m.req.nc);
        rc = igks_get_fields(c.ctx, m.sid, W.data());
        if (rc) return ctx_fail(s, c.ctx, rc, "reading fields");
        s->fields[r.id] = std::move(W);
      }
      r.t_finish = now_s(s);
      m.live = false;
      // the host copy of the mesh is no longer needed
      m.req.xy = {}; m.req.cell_ptr = {}; m.req.cell_nodes = {};
      m.req.face_nodes = {}; m.req.face_cells = {}; m.req.face_bc = {};
      s->done.push_back(r);
    }
  }
  std::vector<Cohort> keep;
  for (Cohort& c : s->cohorts) {
    if (live_cells(c) == 0) {
      igks_destroy(c.ctx);
      continue;
    }
    keep.push_back(std::move(c));
  }
  s->cohorts.swap(keep);
  return 0;
}

static void fill_status(const igks_server* s, igks_server_status* st) {
  if (!st) return;
  *st = igks_server_status{};
  st->queued = (int32_t)s->queue.size();
  st->live = n_live(s);
  st->cohorts = (int32_t)s->cohorts.size();
  st->finished = (int32_t)s->done.size();
  st->bytes = resident_bytes(s);
  st->budget = s->opt.hbm_budget;
  st->admitted = s->last_admitted;
  st->repacked = s->last_repacked;
  st->step_s = s->last_step;
}

extern "C" {

int igks_server_create(const igks_server_options* opt, igks_server** out) {
  if (!opt || !out) return IGKS_EINVAL;
  *out = nullptr;
  if ((opt->precision != IGKS_PREC_FP64 && opt->precision != IGKS_PREC_MIXED && opt->precision != IGKS_PREC_DF64) ||
      opt->max_slots < 1 ||
      opt->max_cohort < 1 || opt->iters_per_step < 1 || opt->max_iters < 1 || opt->hbm_budget < 0 ||
      !(opt->repack_fraction >= 0.0 && opt->repack_fraction <= 1.0))
    return IGKS_EINVAL;
  if (cudaSetDevice(opt->device) != cudaSuccess) return IGKS_ECUDA;
  igks_server* s = new igks_server();
  s->opt = *opt;
  if (s->opt.hbm_budget == 0) {
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
      delete s;
      return IGKS_ECUDA;
    }
    s->opt.hbm_budget = (int64_t)(0.9 * (double)fr);
  }
  s->t0 = std::chrono::steady_clock::now();
  *out = s;
  return IGKS_OK;
}

int igks_server_submit(igks_server* s, const igks_request* q, int64_t* id) {
  if (!s || !q) return IGKS_EINVAL;
  std::string msg;
  int rc = igks_check_mesh_(q->n_nodes, q->xy, q->n_cells, q->cell_ptr, q->cell_nodes, q->n_faces, q->face_nodes,
                            q->face_cells, q->face_bc, &msg);
  if (rc) return sfail(s, rc, msg);
  if (!igks_check_flow_(&q->flow)) return sfail(s, IGKS_EINVAL, "invalid flow conditions");
  Request r;
  r.nn = q->n_nodes; r.nc = q->n_cells; r.nf = q->n_faces;
  const int nk = q->cell_ptr[q->n_cells];
  igks_footprint_bytes(r.nn, r.nc, r.nf, nk, &r.footprint);
  if (r.footprint > s->opt.hbm_budget) return sfail(s, IGKS_ENOMEM, "request larger than the HBM budget");
  r.xy.assign(q->xy, q->xy + 2 * (size_t)r.nn);
  r.cell_ptr.assign(q->cell_ptr, q->cell_ptr + r.nc + 1);
  r.cell_nodes.assign(q->cell_nodes, q->cell_nodes + nk);
  r.face_nodes.assign(q->face_nodes, q->face_nodes + 2 * (size_t)r.nf);
  r.face_cells.assign(q->face_cells, q->face_cells + 2 * (size_t)r.nf);
  r.face_bc.assign(q->face_bc, q->face_bc + r.nf);
  if (q->W0) {
    for (int i = 0; i < r.nc; i++)
      if (!(q->W0[i] > 0.0) || !std::isfinite(q->W0[3 * (size_t)r.nc + i]))
        return sfail(s, IGKS_EINVAL, "non-physical starting state");
    r.W0.assign(q->W0, q->W0 + 5 * (size_t)r.nc);
  }
  r.flow = q->flow;
  r.tag = q->tag;
  r.id = s->next_id++;
  r.t_submit = now_s(s);
  s->queue.push_back(std::move(r));
  if (id) *id = s->queue.back().id;
  return IGKS_OK;
}

int igks_server_step(igks_server* s, igks_server_status* status) {
  if (!s) return IGKS_EINVAL;
  const double t = now_s(s);
  s->last_admitted = s->last_repacked = 0;
  int rc = admit(s);
  if (!rc) rc = run(s);
  if (!rc) rc = retire(s);
  s->last_step = now_s(s) - t;
  fill_status(s, status);
  return rc;
}

int igks_server_poll(igks_server* s, igks_result* out, int32_t cap, int32_t* n) {
  if (!s || !n || cap < 0 || (cap > 0 && !out)) return IGKS_EINVAL;
  int k = 0;
  while (k < cap && !s->done.empty()) {
    out[k++] = s->done.front();
    s->done.pop_front();
  }
  *n = k;
  return IGKS_OK;
}

int igks_server_take_fields(igks_server* s, int64_t id, double* W) {
  if (!s || !W) return IGKS_EINVAL;
  auto it = s->fields.find(id);
  if (it == s->fields.end()) return sfail(s, IGKS_EINVAL, "no kept fields for this id");
  std::copy(it->second.begin(), it->second.end(), W);
  s->fields.erase(it);
  return IGKS_OK;
}

int igks_server_now(igks_server* s, double* t) {
  if (!s || !t) return IGKS_EINVAL;
  *t = now_s(s);
  return IGKS_OK;
}

int igks_server_get_status(igks_server* s, igks_server_status* status) {
  if (!s || !status) return IGKS_EINVAL;
  fill_status(s, status);
  return IGKS_OK;
}

int igks_server_destroy(igks_server* s) {
  if (!s) return IGKS_EINVAL;
  for (Cohort& c : s->cohorts)
    if (c.ctx) igks_destroy(c.ctx);
  delete s;
  return IGKS_OK;
}

const char* igks_server_last_error(igks_server* s) {
  return s ? s->err.c_str() : "null server";
}

}  // extern "C"
