// Serving layer: continuous batching of point-source solves over cached
// per-(model, frequency) factorisations under an HBM budget.  See include/hz.h.
//
// Two native threads share the device:
//   loader  - analyses a problem once (host), makes it resident (device setup and
//             hz_factor on the problem's own stream), evicting least recently used
//             idle problems when the budget requires it;
//   solver  - fills the free slots of every resident problem from its queue, issues
//             one slot-engine step on every busy problem's stream, then completes
//             them in turn, so steps of different problems overlap on the device.
// Requests are served first come, first served within a problem; each source is one
// slot (one right-hand side of the pseudo-block FGMRES), so a request's sources can
// finish in any order and share steps with other requests' sources.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "../../include/hz.h"
#include "engine.h"
#include "host.h"

namespace {

using clk = std::chrono::steady_clock;

enum { P_IDLE = 0, P_LOADING = 1, P_READY = 2 };

struct Problem {
  int id = 0;
  double freq = 0;
  int order = 1;
  hz_options opt{};
  // owned copy of the mesh description
  std::vector<double> xyz, c_re, c_im, cxyz;
  std::vector<int32_t> tets, faces, ctets, cfaces, parent, part;
  std::vector<int8_t> tag, ctag;
  hz_mesh_desc md{};
  std::unique_ptr<hz::HostProblem> host;     // analysis, kept after the first use
  int64_t est_persistent = 0, est_transient = 0;
  int64_t n = -1;
  hz_ctx* ctx = nullptr;
  cudaStream_t stream = nullptr;
  int state = P_IDLE;
  int64_t bytes = 0;                          // resident bytes (or reservation while loading)
  double last_use = 0;
  std::deque<uint64_t> queue;                 // requests with sources not yet admitted
  int inflight = 0;                           // sources admitted and not yet harvested
  std::vector<std::pair<uint64_t, int>> owner;   // slot -> (request, source)
};

struct Request {
  uint64_t id = 0;
  int problem = 0;
  double tol = 0;
  int nsrc = 0;
  std::vector<double> src;
  int next = 0, finished = 0;
  std::vector<double> x;                      // interleaved complex, n * nsrc
  std::vector<hz_rhs_info> info;
  hz_request_times t{};
  bool done = false;
};

int64_t free_device_bytes() {
  size_t fr = 0, tot = 0;
  if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return int64_t(fr);
}

}  // namespace

struct hz_server {
  hz_server_options opt{};
  int64_t budget = 0;
  clk::time_point t0 = clk::now();
  std::mutex mu;
  std::condition_variable cv_solver, cv_loader, cv_done;
  bool stop = false;
  std::vector<std::unique_ptr<Problem>> problems;
  std::map<uint64_t, std::unique_ptr<Request>> requests;
  uint64_t next_id = 1;
  int64_t resident = 0;
  hz_server_stats st{};
  std::vector<double> latencies;
  double first_submit = -1, last_done = 0;
  std::string err;
  long long launches0 = 0;
  std::thread solver, loader;

  double now() const { return std::chrono::duration<double>(clk::now() - t0).count(); }
  void solver_loop();
  void loader_loop();
  void finish_source(Request& r, int src, const hz_rhs_info& info);   // under mu
  void fail_queued(Problem& p, hz_status s);                          // under mu
};

// Records one finished source of request r; completes the request when all are in.
void hz_server::finish_source(Request& r, int src, const hz_rhs_info& info) {
  r.info[size_t(src)] = info;
  r.finished++;
  st.rhs_done++;
  if (info.status != HZ_OK && r.t.status == HZ_OK) r.t.status = info.status;
  if (r.finished == r.nsrc) {
    r.done = true;
    r.t.done_s = now();
    r.t.latency_s = r.t.done_s - r.t.submit_s;
    latencies.push_back(r.t.latency_s);
    last_done = r.t.done_s;
    st.requests_done++;
    cv_done.notify_all();
  }
}

// Ends every queued source of p with status s (the problem cannot be made resident).
void hz_server::fail_queued(Problem& p, hz_status s) {
  while (!p.queue.empty()) {
    auto it = requests.find(p.queue.front());
    p.queue.pop_front();
    if (it == requests.end()) continue;
    Request& r = *it->second;
    if (r.t.admit_s == 0) r.t.admit_s = now();
    while (r.next < r.nsrc) {
      hz_rhs_info inf{0, int32_t(s), NAN};
      finish_source(r, r.next++, inf);
    }
  }
}

void hz_server::loader_loop() {
  cudaSetDevice(opt.device);
  for (;;) {
    Problem* p = nullptr;
    {
      std::unique_lock<std::mutex> lk(mu);
      for (;;) {
        if (stop) return;
        double oldest = 1e300;
        p = nullptr;
        for (auto& q : problems) {
          if (q->state != P_IDLE || q->queue.empty()) continue;
          const double ts = requests.at(q->queue.front())->t.submit_s;
          if (ts < oldest) {
            oldest = ts;
            p = q.get();
          }
        }
        if (p) break;
        cv_loader.wait_for(lk, std::chrono::milliseconds(100));
      }
      p->state = P_LOADING;
    }
    // host analysis, once per problem
    if (!p->host) {
      auto P = std::make_unique<hz::HostProblem>();
      std::string e;
      const auto ta = clk::now();
      hz_status s = hz_engine::analyse_problem(&p->md, &p->opt, *P, e);
      std::lock_guard<std::mutex> lk(mu);
      st.factor_seconds += std::chrono::duration<double>(clk::now() - ta).count();
      if (s != HZ_OK) {
        err = "problem " + std::to_string(p->id) + ": " + e;
        p->state = P_IDLE;
        fail_queued(*p, s);
        continue;
      }
      p->host = std::move(P);
      p->n = p->host->dofs.n;
      hz_engine::plan_bytes(*p->host, p->opt, p->est_persistent, p->est_transient);
      st.analyses++;
    }
    // room under the budget: evict idle problems, least recently used first.  A problem
    // that needs more than the whole budget can never be admitted, whatever else is
    // resident: its requests fail at once (waiting for others to leave would never end
    // when they stay resident and idle).
    const int64_t need = p->est_persistent + p->est_transient;
    std::vector<Problem*> evict;
    if (budget > 0 && need > budget) {
      std::lock_guard<std::mutex> lk(mu);
      err = "problem " + std::to_string(p->id) + " needs " + std::to_string(need) + " bytes, over the budget of " +
            std::to_string(budget);
      p->state = P_IDLE;
      fail_queued(*p, HZ_ERR_OOM);
      cv_done.notify_all();
      continue;
    }
    {
      std::unique_lock<std::mutex> lk(mu);
      for (;;) {
        if (stop) {
          p->state = P_IDLE;
          return;
        }
        std::vector<int64_t> bytes;
        std::vector<double> last;
        std::vector<int32_t> ok;
        std::vector<Problem*> cand;
        for (auto& q : problems) {
          if (q->state != P_READY) continue;
          cand.push_back(q.get());
          bytes.push_back(q->bytes);
          last.push_back(q->last_use);
          ok.push_back(q->inflight == 0 && q->queue.empty() ? 1 : 0);
        }
        std::vector<int32_t> sel(cand.size() + 1);
        const int32_t k = hz_select_evictions(int32_t(cand.size()), bytes.data(), last.data(), ok.data(), resident,
                                              need, budget, sel.data());
        if (k >= 0) {
          for (int32_t q = 0; q < k; q++) {
            Problem* v = cand[size_t(sel[size_t(q)])];
            v->state = P_IDLE;
            resident -= v->bytes;
            v->bytes = 0;
            evict.push_back(v);
          }
          resident += need;                   // reservation while loading
          p->bytes = need;
          break;
        }
        bool any_ready = false;
        for (auto& q : problems) any_ready = any_ready || q->state == P_READY || (q.get() != p && q->state == P_LOADING);
        if (!any_ready) {                     // does not fit even on an empty device
          err = "problem " + std::to_string(p->id) + " needs " + std::to_string(need) + " bytes, over the budget";
          p->state = P_IDLE;
          fail_queued(*p, HZ_ERR_OOM);
          p = nullptr;
          break;
        }
        cv_loader.wait_for(lk, std::chrono::milliseconds(50));
      }
    }
    for (Problem* v : evict) {
      hz_free(v->ctx);
      v->ctx = nullptr;
      if (v->stream) cudaStreamDestroy(v->stream);
      v->stream = nullptr;
      std::lock_guard<std::mutex> lk(mu);
      st.evictions++;
    }
    if (!p) continue;
    // device setup and factorisation on the problem's own stream
    const auto tf = clk::now();
    hz_status s = HZ_OK;
    std::string e;
    hz_ctx* ctx = nullptr;
    cudaStream_t stream = nullptr;
    if (cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      s = HZ_ERR_CUDA;
      e = "cudaStreamCreate failed";
    }
    if (s == HZ_OK) {
      hz_options o = p->opt;
      o.stream = reinterpret_cast<uintptr_t>(stream);
      o.hbm_budget = budget > 0 ? uint64_t(std::max<int64_t>(need, 1)) : 0;
      s = hz_engine::create(*p->host, p->order, &o, &ctx, e);
    }
    if (s == HZ_OK) {
      s = hz_factor(ctx, p->freq);
      if (s != HZ_OK) e = hz_last_error(ctx);
    }
    std::lock_guard<std::mutex> lk(mu);
    st.factor_seconds += std::chrono::duration<double>(clk::now() - tf).count();
    resident -= p->bytes;
    p->bytes = 0;
    if (s != HZ_OK) {
      if (ctx) hz_free(ctx);
      if (stream) cudaStreamDestroy(stream);
      err = "problem " + std::to_string(p->id) + ": " + e;
      p->state = P_IDLE;
      fail_queued(*p, s);
      continue;
    }
    st.factorisations++;
    p->ctx = ctx;
    p->stream = stream;
    p->bytes = hz_engine::device_bytes(ctx);
    p->owner.assign(size_t(hz_engine::slot_count(ctx)), {0, -1});
    p->last_use = now();
    resident += p->bytes;
    st.peak_resident_bytes = std::max(st.peak_resident_bytes, resident);
    p->state = P_READY;
    cv_solver.notify_all();
  }
}

void hz_server::solver_loop() {
  cudaSetDevice(opt.device);
  struct Admit {
    Problem* p;
    int slot;
    Request* r;
    int src;
  };
  for (;;) {
    std::vector<Problem*> busy;
    std::vector<Admit> admits;
    {
      std::unique_lock<std::mutex> lk(mu);
      for (;;) {
        if (stop) return;
        busy.clear();
        for (auto& q : problems)
          if (q->state == P_READY && (q->inflight > 0 || !q->queue.empty())) busy.push_back(q.get());
        if (!busy.empty()) break;
        cv_solver.wait_for(lk, std::chrono::milliseconds(50));
      }
      // fill free slots first come, first served
      for (Problem* p : busy) {
        const int S = int(p->owner.size());
        for (int i = 0; i < S && !p->queue.empty(); i++) {
          if (p->owner[size_t(i)].second >= 0) continue;
          Request& r = *requests.at(p->queue.front());
          if (r.t.admit_s == 0) r.t.admit_s = now();
          if (r.x.empty()) r.x.assign(size_t(2) * size_t(p->n) * size_t(r.nsrc), 0.0);
          admits.push_back({p, i, &r, r.next});
          p->owner[size_t(i)] = {r.id, r.next};
          p->inflight++;
          if (++r.next == r.nsrc) p->queue.pop_front();
        }
      }
    }
    for (const Admit& a : admits) {
      hz_status s = hz_engine::slot_point_source(a.p->ctx, a.slot, a.r->src.data() + 3 * a.src);
      if (s == HZ_OK) s = hz_engine::slot_start(a.p->ctx, a.slot, a.r->tol, a.src);
      if (s != HZ_OK) {
        std::lock_guard<std::mutex> lk(mu);
        err = hz_last_error(a.p->ctx);
        hz_engine::slot_reset(a.p->ctx, a.slot);
        a.p->owner[size_t(a.slot)] = {0, -1};
        a.p->inflight--;
        finish_source(*a.r, a.src, hz_rhs_info{0, int32_t(s), NAN});
      }
    }
    for (Problem* p : busy)
      if (hz_engine::slots_running(p->ctx)) hz_engine::slots_issue(p->ctx);
    for (Problem* p : busy) {
      hz_status s = HZ_OK;
      if (hz_engine::slots_running(p->ctx)) s = hz_engine::slots_complete(p->ctx);
      const int S = int(p->owner.size());
      for (int i = 0; i < S; i++) {
        const int state = hz_engine::slot_state(p->ctx, i);
        if (p->owner[size_t(i)].second < 0) continue;
        if (state != hz_engine::SLOT_DONE && s == HZ_OK) continue;
        const auto own = p->owner[size_t(i)];
        Request* r = nullptr;
        {
          std::lock_guard<std::mutex> lk(mu);
          r = requests.at(own.first).get();
        }
        hz_rhs_info inf{0, int32_t(s), NAN};
        if (state != hz_engine::SLOT_DONE) hz_engine::slot_reset(p->ctx, i);   // step failed
        if (state == hz_engine::SLOT_DONE) {
          hz_status h = hz_engine::slot_harvest(p->ctx, i, r->x.data() + size_t(2) * size_t(p->n) * size_t(own.second),
                                                false, &inf);
          if (h != HZ_OK) inf = hz_rhs_info{0, int32_t(h), NAN};
        }
        std::lock_guard<std::mutex> lk(mu);
        p->owner[size_t(i)] = {0, -1};
        p->inflight--;
        p->last_use = now();
        finish_source(*r, own.second, inf);
        cv_loader.notify_all();
      }
      std::lock_guard<std::mutex> lk(mu);
      st.steps++;
    }
  }
}

extern "C" {

int32_t hz_select_evictions(int32_t count, const int64_t* bytes, const double* last_use, const int32_t* evictable,
                            int64_t resident, int64_t need, int64_t budget, int32_t* out) {
  if (count < 0 || need < 0 || resident < 0 || (count > 0 && (!bytes || !last_use || !evictable || !out))) return -1;
  if (budget <= 0 || resident + need <= budget) return 0;
  std::vector<int32_t> order;
  for (int32_t i = 0; i < count; i++)
    if (evictable[i]) order.push_back(i);
  std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) { return last_use[a] < last_use[b]; });
  int64_t have = resident;
  int32_t k = 0;
  for (int32_t i : order) {
    if (have + need <= budget) break;
    out[k++] = i;
    have -= bytes[i];
  }
  return have + need <= budget ? k : -1;
}

hz_status hz_server_create(const hz_server_options* opt, hz_server** out) {
  if (!opt || !out) return HZ_ERR_ARG;
  *out = nullptr;
  if (opt->slots < 2 || opt->slots > 16 || (opt->precision != HZ_FP64 && opt->precision != HZ_MIXED))
    return HZ_ERR_ARG;
  if (cudaSetDevice(opt->device) != cudaSuccess) {
    cudaGetLastError();
    return HZ_ERR_CUDA;
  }
  hz_server* s = new hz_server();
  s->opt = *opt;
  s->launches0 = hz::launch_count();
  s->budget = opt->hbm_budget ? int64_t(opt->hbm_budget) : std::max<int64_t>(free_device_bytes() - (int64_t(2) << 30), 1);
  s->solver = std::thread([s] { s->solver_loop(); });
  s->loader = std::thread([s] { s->loader_loop(); });
  *out = s;
  return HZ_OK;
}

hz_status hz_server_add_problem(hz_server* s, const hz_mesh_desc* md, const hz_options* op, double freq_hz,
                                int32_t* problem_id) {
  if (!s || !md || !op || !problem_id || !(freq_hz > 0.0) || !std::isfinite(freq_hz)) return HZ_ERR_ARG;
  if (md->nv <= 0 || md->ne <= 0 || !md->xyz || !md->tets || !md->c_re || !md->c_im) return HZ_ERR_ARG;
  if (md->nf > 0 && (!md->faces || !md->face_tag)) return HZ_ERR_ARG;
  auto p = std::make_unique<Problem>();
  p->freq = freq_hz;
  p->order = md->order;
  p->opt = *op;
  p->opt.precision = s->opt.precision;
  p->opt.block_size = s->opt.slots;
  p->opt.recycle = 0;                       // slots run pseudo-block FGMRES
  p->xyz.assign(md->xyz, md->xyz + 3 * md->nv);
  p->tets.assign(md->tets, md->tets + 4 * md->ne);
  p->c_re.assign(md->c_re, md->c_re + md->ne);
  p->c_im.assign(md->c_im, md->c_im + md->ne);
  if (md->nf > 0) {
    p->faces.assign(md->faces, md->faces + 3 * md->nf);
    p->tag.assign(md->face_tag, md->face_tag + md->nf);
  }
  p->md = *md;
  p->md.xyz = p->xyz.data();
  p->md.tets = p->tets.data();
  p->md.c_re = p->c_re.data();
  p->md.c_im = p->c_im.data();
  p->md.faces = p->faces.data();
  p->md.face_tag = p->tag.data();
  if (op->levels == 2) {
    if (!md->coarse_xyz || !md->coarse_tets || !md->fine_parent || md->coarse_nv <= 0 || md->coarse_ne <= 0)
      return HZ_ERR_ARG;
    p->cxyz.assign(md->coarse_xyz, md->coarse_xyz + 3 * md->coarse_nv);
    p->ctets.assign(md->coarse_tets, md->coarse_tets + 4 * md->coarse_ne);
    if (md->coarse_nf > 0) {
      p->cfaces.assign(md->coarse_faces, md->coarse_faces + 3 * md->coarse_nf);
      p->ctag.assign(md->coarse_face_tag, md->coarse_face_tag + md->coarse_nf);
    }
    p->parent.assign(md->fine_parent, md->fine_parent + md->ne);
    p->md.coarse_xyz = p->cxyz.data();
    p->md.coarse_tets = p->ctets.data();
    p->md.coarse_faces = p->cfaces.data();
    p->md.coarse_face_tag = p->ctag.data();
    p->md.fine_parent = p->parent.data();
  }
  if (op->elem_part) {
    p->part.assign(op->elem_part, op->elem_part + md->ne);
    p->opt.elem_part = p->part.data();
  }
  std::lock_guard<std::mutex> lk(s->mu);
  p->id = int32_t(s->problems.size());
  *problem_id = p->id;
  s->problems.push_back(std::move(p));
  return HZ_OK;
}

hz_status hz_server_submit(hz_server* s, int32_t problem_id, const double* src_xyz, int32_t nsrc, double tol,
                           uint64_t* request_id) {
  if (!s || !request_id || nsrc < 0 || (nsrc > 0 && !src_xyz) || !(tol > 0.0)) return HZ_ERR_ARG;
  auto r = std::make_unique<Request>();
  r->problem = problem_id;
  r->tol = tol;
  r->nsrc = nsrc;
  r->src.assign(src_xyz, src_xyz + 3 * int64_t(nsrc));
  r->info.assign(size_t(nsrc), hz_rhs_info{0, HZ_OK, 0.0});
  std::lock_guard<std::mutex> lk(s->mu);
  if (problem_id < 0 || problem_id >= int32_t(s->problems.size())) return HZ_ERR_ARG;
  Problem& p = *s->problems[size_t(problem_id)];
  r->id = s->next_id++;
  r->t.nsrc = nsrc;
  r->t.submit_s = s->now();
  if (s->first_submit < 0) s->first_submit = r->t.submit_s;
  *request_id = r->id;
  Request& ref = *r;
  s->requests[r->id] = std::move(r);
  if (nsrc == 0) {
    ref.done = true;
    ref.t.admit_s = ref.t.done_s = ref.t.submit_s;
    s->cv_done.notify_all();
    return HZ_OK;
  }
  // the result buffer is sized once the problem's dof count is known (first analysis)
  p.queue.push_back(ref.id);
  s->cv_loader.notify_all();
  s->cv_solver.notify_all();
  return HZ_OK;
}

hz_status hz_server_wait(hz_server* s, uint64_t request_id, double timeout_s, hz_request_times* times) {
  if (!s) return HZ_ERR_ARG;
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->requests.find(request_id);
  if (it == s->requests.end()) return HZ_ERR_ARG;
  Request& r = *it->second;
  const auto until =
      clk::now() + std::chrono::duration_cast<clk::duration>(std::chrono::duration<double>(timeout_s > 0 ? timeout_s : 1e9));
  while (!r.done)
    if (s->cv_done.wait_until(lk, until) == std::cv_status::timeout && !r.done) break;
  if (times) *times = r.t;
  return r.done ? HZ_OK : HZ_ERR_TIMEOUT;
}

hz_status hz_server_collect(hz_server* s, uint64_t request_id, void* x, hz_rhs_info* info, hz_request_times* times) {
  if (!s) return HZ_ERR_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->requests.find(request_id);
  if (it == s->requests.end()) return HZ_ERR_ARG;
  Request& r = *it->second;
  if (!r.done) return HZ_ERR_STATE;
  if (x && !r.x.empty()) std::memcpy(x, r.x.data(), r.x.size() * sizeof(double));
  if (info && r.nsrc > 0) std::memcpy(info, r.info.data(), size_t(r.nsrc) * sizeof(hz_rhs_info));
  if (times) *times = r.t;
  const hz_status worst = hz_status(r.t.status);
  s->requests.erase(it);
  return worst;
}

int64_t hz_server_ndofs(hz_server* s, int32_t problem_id) {
  if (!s) return -1;
  std::lock_guard<std::mutex> lk(s->mu);
  if (problem_id < 0 || problem_id >= int32_t(s->problems.size())) return -1;
  return s->problems[size_t(problem_id)]->n;
}

hz_status hz_server_get_stats(hz_server* s, hz_server_stats* out) {
  if (!s || !out) return HZ_ERR_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  *out = s->st;
  std::vector<double> l = s->latencies;
  std::sort(l.begin(), l.end());
  auto rank = [&](double q) {
    if (l.empty()) return 0.0;
    const size_t k = size_t(std::ceil(q * double(l.size())));
    return l[std::min(l.size(), std::max<size_t>(k, 1)) - 1];
  };
  out->p50_latency_s = rank(0.50);
  out->p99_latency_s = rank(0.99);
  const double span = s->last_done - s->first_submit;
  out->rhs_per_s = span > 0 ? double(s->st.rhs_done) / span : 0.0;
  out->resident_bytes = s->resident;
  out->budget_bytes = s->budget;
  out->launches = hz::launch_count() - s->launches0;
  return HZ_OK;
}

const char* hz_server_last_error(hz_server* s) {
  if (!s) return "null server";
  std::lock_guard<std::mutex> lk(s->mu);
  static thread_local std::string copy;
  copy = s->err;
  return copy.c_str();
}

void hz_server_free(hz_server* s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv_solver.notify_all();
  s->cv_loader.notify_all();
  s->cv_done.notify_all();
  if (s->solver.joinable()) s->solver.join();
  if (s->loader.joinable()) s->loader.join();
  for (auto& p : s->problems) {
    hz_free(p->ctx);
    if (p->stream) cudaStreamDestroy(p->stream);
  }
  delete s;
}

}  // extern "C"
