// Serving runtime: continuous batching of solve requests on one GPU.
//
// The imaging loop of Sec. 6 needs one direct Maxwell solve per antenna and per permittivity
// update; requests of different meshes, degrees and right-hand-side counts arrive while others
// run.  A request goes through three stages:
//   1. planning (host threads): the mesh set-up of oras_create (topology, DOF map, partition,
//      overlap, CSR pattern) runs on the host, which fixes the request's device footprint
//      (factor arena, matrices, Krylov basis of k right-hand sides);
//   2. admission (first in, first out): the oldest planned request is admitted as soon as a
//      worker slot is free and its footprint fits in the HBM budget next to the requests already
//      on the GPU; a request larger than the whole budget is rejected;
//   3. execution (one host worker thread and one CUDA stream per slot): assembly, batched LU and
//      FGMRES of the request run on the slot's stream, so the kernels of the admitted requests
//      overlap on the device; stream-ordered allocation keeps one request's frees from
//      synchronising the others.  The factors and the Krylov basis stay resident for the whole
//      solve and are released when the request finishes, which frees budget for the queue.
// Each request computes exactly what oras_setup + oras_solve compute for it alone: the kernels
// of a request depend only on its own buffers.
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>

#include "internal.h"

using namespace oras;
int64_t footprint_bytes(const oras_handle* h, int k);  // api.cpp

namespace {

struct Request {
  int64_t ticket = 0;
  std::vector<double> xyz, dipoles, beta;
  std::vector<uint8_t> face_kind;
  std::vector<int32_t> tets, part;
  std::vector<oras_complex> eps, mu, rhs;
  oras_problem prob{};
  oras_options opt{};
  bool has_opt = false;
  int k = 1;
  double tol = 1e-8;
  int64_t n_rhs_rows = 0;
  oras_handle* h = nullptr;
  std::vector<oras_complex> x;
  std::vector<oras_info> info;
  oras_ticket rec{};
  std::string err;
  enum State { QUEUED, PLANNED, RUNNING, DONE } state = QUEUED;
};

double seconds_since(std::chrono::steady_clock::time_point t0) {
  return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
}

}  // namespace

struct oras_server {
  oras_server_config cfg{};
  std::mutex mu;
  std::condition_variable cv;            // every state change
  std::deque<Request*> plan_q;           // submitted, host set-up pending
  std::deque<Request*> ready_q;          // planned, in ticket order, waiting for admission
  std::map<int64_t, Request*> live;      // not yet collected by oras_wait
  std::map<int64_t, oras_ticket> done;   // collected tickets
  std::map<int64_t, std::string> errors; // messages of failed tickets
  int64_t next_ticket = 1;
  oras_server_counters st{};
  bool stop = false;
  std::vector<std::thread> planners, workers;
  std::chrono::steady_clock::time_point t0 = std::chrono::steady_clock::now();
  std::string err;
};

namespace {

void finish_locked(oras_server* S, Request* q, int status, const std::string& err) {
  q->rec.status = status;
  q->rec.done_s = seconds_since(S->t0);
  q->err = err;
  if (!err.empty()) S->errors[q->ticket] = err;
  q->state = Request::DONE;
  if (status == ORAS_ERR_REJECTED) ++S->st.rejected;
  else ++S->st.completed;
}

void planner_main(oras_server* S) {
  for (;;) {
    Request* q = nullptr;
    {
      std::unique_lock<std::mutex> lk(S->mu);
      S->cv.wait(lk, [&] { return S->stop || !S->plan_q.empty(); });
      if (S->stop) return;
      q = S->plan_q.front();
      S->plan_q.pop_front();
    }
    oras_handle* h = nullptr;
    int rc = oras_create(&q->prob, q->has_opt ? &q->opt : nullptr, &h);
    std::string err = rc ? std::string(oras_last_error(nullptr)) : std::string();
    int64_t fp = 0, N = 0;
    if (rc == ORAS_OK) {
      N = oras_ndof(h);
      if (!q->rhs.empty() && q->n_rhs_rows != N) {
        rc = ORAS_ERR_INVALID_ARG;
        err = "oras_submit: rhs has " + std::to_string(q->n_rhs_rows) + " rows, the problem has " +
              std::to_string(N) + " DOFs";
      } else {
        // dipole requests also hold the right-hand sides and the solution on the device
        fp = footprint_bytes(h, q->k) + (q->dipoles.empty() ? 0 : 2 * N * q->k * 16 + (4 << 20));
        if (fp > S->cfg.hbm_budget) {
          rc = ORAS_ERR_REJECTED;
          err = "oras_submit: the request needs " + std::to_string(fp) + " device bytes, more than the budget of " +
                std::to_string(S->cfg.hbm_budget);
        }
      }
      if (rc != ORAS_OK) {
        oras_destroy(h);
        h = nullptr;
      }
    }
    {
      std::lock_guard<std::mutex> lk(S->mu);
      q->rec.planned_s = seconds_since(S->t0);
      q->rec.footprint = fp;
      q->rec.ndof = N;
      if (rc == ORAS_OK && S->stop) {
        oras_destroy(h);
        rc = ORAS_ERR_STATE;
        err = "server destroyed before the request was admitted";
      }
      if (rc != ORAS_OK) {
        finish_locked(S, q, rc, err);
      } else {
        q->h = h;
        q->state = Request::PLANNED;
        auto it = S->ready_q.begin();
        while (it != S->ready_q.end() && (*it)->ticket < q->ticket) ++it;
        S->ready_q.insert(it, q);
      }
    }
    S->cv.notify_all();
  }
}

// Runs factorisation and solve of an admitted request on `stream`; returns its status.
int run_request(Request* q, cudaStream_t stream, std::string& err) {
  oras_handle* h = q->h;
  oras_set_stream(h, stream);
  const int64_t N = oras_ndof(h);
  q->x.assign((size_t)N * q->k, oras_complex{0.0, 0.0});
  q->info.assign(q->k, oras_info{});
  int rc = oras_factor(h, q->prob.eps_r, q->prob.mu_r, q->prob.k0, ORAS_MEM_HOST);
  if (rc == ORAS_OK) {
    if (q->dipoles.empty()) {
      rc = oras_solve(h, q->rhs.data(), q->k, q->tol, q->x.data(), q->info.data(), ORAS_MEM_HOST);
    } else {
      // right-hand sides w_i(x0) . dir evaluated on the device, solved there, x copied back
      oras_complex* b = nullptr;
      oras_complex* xd = nullptr;
      const size_t bytes = (size_t)N * q->k * sizeof(oras_complex);
      cudaError_t e = pool_malloc((void**)&b, bytes, stream);
      if (e == cudaSuccess) e = pool_malloc((void**)&xd, bytes, stream);
      if (e != cudaSuccess) {
        rc = e == cudaErrorMemoryAllocation ? ORAS_ERR_OUT_OF_MEMORY : ORAS_ERR_CUDA;
        err = std::string("right-hand side buffers: ") + cudaGetErrorString(e);
      }
      for (int j = 0; j < q->k && rc == ORAS_OK; ++j)
        rc = oras_rhs_dipole(h, &q->dipoles[6 * j], &q->dipoles[6 * j + 3], b + (size_t)N * j, ORAS_MEM_DEVICE);
      if (rc == ORAS_OK) rc = oras_solve(h, b, q->k, q->tol, xd, q->info.data(), ORAS_MEM_DEVICE);
      if (rc == ORAS_OK || rc == ORAS_NOT_CONVERGED) {
        e = cudaMemcpyAsync(q->x.data(), xd, bytes, cudaMemcpyDeviceToHost, stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
        if (e != cudaSuccess) {
          rc = ORAS_ERR_CUDA;
          err = std::string("copy of the solution: ") + cudaGetErrorString(e);
        }
      }
      if (b) cudaFreeAsync(b, stream);
      if (xd) cudaFreeAsync(xd, stream);
    }
  }
  if (rc != ORAS_OK && err.empty()) err = oras_last_error(h);
  oras_destroy(h);  // frees on the stream and synchronises it
  q->h = nullptr;
  return rc;
}

void worker_main(oras_server* S) {
  bool ready = false;
  cudaStream_t stream = nullptr;
  for (;;) {
    Request* q = nullptr;
    {
      std::unique_lock<std::mutex> lk(S->mu);
      S->cv.wait(lk, [&] {
        return S->stop || (!S->ready_q.empty() && S->st.hbm_in_use + S->ready_q.front()->rec.footprint <= S->cfg.hbm_budget);
      });
      if (S->stop) break;
      q = S->ready_q.front();
      S->ready_q.pop_front();
      S->st.hbm_in_use += q->rec.footprint;
      S->st.hbm_peak = std::max(S->st.hbm_peak, S->st.hbm_in_use);
      ++S->st.active;
      S->st.peak_active = std::max(S->st.peak_active, S->st.active);
      q->state = Request::RUNNING;
      q->rec.admitted_s = seconds_since(S->t0);
    }
    int rc = ORAS_OK;
    std::string err;
    if (!ready) {
      cudaError_t e = cudaSetDevice(S->cfg.device);
      if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking);
      if (e != cudaSuccess) {
        rc = ORAS_ERR_CUDA;
        err = std::string("worker set-up: ") + cudaGetErrorString(e);
      } else {
        ready = true;
      }
    }
    if (rc == ORAS_OK) {
      rc = run_request(q, stream, err);
    } else {
      oras_destroy(q->h);
      q->h = nullptr;
    }
    {
      std::lock_guard<std::mutex> lk(S->mu);
      S->st.hbm_in_use -= q->rec.footprint;
      --S->st.active;
      finish_locked(S, q, rc, err);
    }
    S->cv.notify_all();
  }
  if (stream) cudaStreamDestroy(stream);
}

}  // namespace

extern "C" {

int oras_server_create(const oras_server_config* cfg, oras_server** out) {
  if (!out) return ORAS_ERR_INVALID_ARG;
  *out = nullptr;
  oras_server_config c{};
  if (cfg) c = *cfg;
  if (c.max_active <= 0) c.max_active = 4;
  if (c.planners <= 0) c.planners = 2;
  if (c.max_active > 64 || c.planners > 64 || c.device < 0 || c.hbm_budget < 0) return ORAS_ERR_INVALID_ARG;
  if (c.hbm_budget == 0) {
    int prev = 0;
    size_t fr = 0, tot = 0;
    cudaGetDevice(&prev);
    cudaError_t e = cudaSetDevice(c.device);
    if (e == cudaSuccess) e = pool_trim(c.device);  // the pool's unused memory counts as free
    if (e == cudaSuccess) e = cudaMemGetInfo(&fr, &tot);
    cudaSetDevice(prev);
    if (e != cudaSuccess) return ORAS_ERR_CUDA;
    c.hbm_budget = (int64_t)(0.9 * (double)fr);
  }
  oras_server* S = new (std::nothrow) oras_server();
  if (!S) return ORAS_ERR_OUT_OF_MEMORY;
  S->cfg = c;
  S->st.hbm_budget = c.hbm_budget;
  try {
    for (int i = 0; i < c.planners; ++i) S->planners.emplace_back(planner_main, S);
    for (int i = 0; i < c.max_active; ++i) S->workers.emplace_back(worker_main, S);
  } catch (const std::exception&) {
    {
      std::lock_guard<std::mutex> lk(S->mu);
      S->stop = true;
    }
    S->cv.notify_all();
    for (auto& t : S->planners) t.join();
    for (auto& t : S->workers) t.join();
    delete S;
    return ORAS_ERR_OUT_OF_MEMORY;
  }
  *out = S;
  return ORAS_OK;
}

int64_t oras_submit(oras_server* S, const oras_problem* p, const oras_options* o, const oras_complex* rhs,
                    int64_t n, const double* dipoles, int32_t k, double tol) {
  if (!S || !p || k < 1 || k > MAX_RHS || !(tol > 0.0) || (rhs == nullptr) == (dipoles == nullptr) ||
      (rhs && n <= 0) || p->nv <= 0 || p->nt <= 0 || !p->xyz || !p->tets || !p->eps_r)
    return ORAS_ERR_INVALID_ARG;
  Request* q = new (std::nothrow) Request();
  if (!q) return ORAS_ERR_OUT_OF_MEMORY;
  try {
    q->xyz.assign(p->xyz, p->xyz + 3 * p->nv);
    q->tets.assign(p->tets, p->tets + 4 * p->nt);
    q->eps.assign(p->eps_r, p->eps_r + p->nt);
    if (p->mu_r) q->mu.assign(p->mu_r, p->mu_r + p->nt);
    if (p->part) q->part.assign(p->part, p->part + p->nt);
    if (p->beta_face) q->beta.assign(p->beta_face, p->beta_face + 4 * p->nt);
    if (p->face_kind) q->face_kind.assign(p->face_kind, p->face_kind + 4 * p->nt);
    if (rhs) q->rhs.assign(rhs, rhs + n * k);
    if (dipoles) q->dipoles.assign(dipoles, dipoles + 6 * k);
  } catch (const std::bad_alloc&) {
    delete q;
    return ORAS_ERR_OUT_OF_MEMORY;
  }
  q->prob = *p;
  q->prob.xyz = q->xyz.data();
  q->prob.tets = q->tets.data();
  q->prob.eps_r = q->eps.data();
  q->prob.mu_r = p->mu_r ? q->mu.data() : nullptr;
  q->prob.part = p->part ? q->part.data() : nullptr;
  q->prob.beta_face = p->beta_face ? q->beta.data() : nullptr;
  q->prob.face_kind = p->face_kind ? q->face_kind.data() : nullptr;
  if (o) {
    q->opt = *o;
    q->has_opt = true;
  }
  q->k = k;
  q->tol = tol;
  q->n_rhs_rows = rhs ? n : 0;
  q->rec.k = k;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->stop) {
      delete q;
      return ORAS_ERR_STATE;
    }
    q->ticket = S->next_ticket++;
    q->rec.submit_s = seconds_since(S->t0);
    S->live[q->ticket] = q;
    S->plan_q.push_back(q);
  }
  S->cv.notify_all();
  return q->ticket;
}

int oras_wait(oras_server* S, int64_t ticket, oras_complex* x, int64_t n, oras_info* info, int32_t timeout_ms) {
  if (!S) return ORAS_ERR_INVALID_ARG;
  Request* q = nullptr;
  {
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->live.find(ticket);
    if (it == S->live.end()) {
      const bool retired = S->done.count(ticket) != 0;
      S->err = std::string("oras_wait: ") + (retired ? "already collected" : "unknown") + " ticket " + std::to_string(ticket);
      return retired ? ORAS_ERR_STATE : ORAS_ERR_INVALID_ARG;
    }
    q = it->second;
    auto pred = [&] { return q->state == Request::DONE; };
    if (timeout_ms < 0) S->cv.wait(lk, pred);
    else if (!S->cv.wait_for(lk, std::chrono::milliseconds(timeout_ms), pred)) return ORAS_PENDING;
    const bool has_x = q->rec.status == ORAS_OK || q->rec.status == ORAS_NOT_CONVERGED;
    if (x && has_x && n != q->rec.ndof) {
      S->err = "oras_wait: x has " + std::to_string(n) + " rows, the problem has " + std::to_string(q->rec.ndof);
      return ORAS_ERR_INVALID_ARG;
    }
    S->live.erase(it);
    S->done[ticket] = q->rec;
  }
  const int status = q->rec.status;
  if (status == ORAS_OK || status == ORAS_NOT_CONVERGED) {
    if (x) std::memcpy(x, q->x.data(), q->x.size() * sizeof(oras_complex));
    if (info) std::memcpy(info, q->info.data(), q->info.size() * sizeof(oras_info));
  }
  delete q;
  return status;
}

int oras_ticket_wait(oras_server* S, int64_t ticket, int32_t timeout_ms) {
  if (!S) return ORAS_ERR_INVALID_ARG;
  std::unique_lock<std::mutex> lk(S->mu);
  auto it = S->live.find(ticket);
  if (it == S->live.end()) return S->done.count(ticket) ? ORAS_OK : ORAS_ERR_INVALID_ARG;
  Request* q = it->second;
  auto pred = [&] { return q->state == Request::DONE; };
  if (timeout_ms < 0) S->cv.wait(lk, pred);
  else if (!S->cv.wait_for(lk, std::chrono::milliseconds(timeout_ms), pred)) return ORAS_PENDING;
  return ORAS_OK;
}

int oras_ticket_info(oras_server* S, int64_t ticket, oras_ticket* out) {
  if (!S || !out) return ORAS_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(S->mu);
  auto it = S->live.find(ticket);
  if (it != S->live.end()) {
    *out = it->second->rec;
    if (it->second->state != Request::DONE) out->status = ORAS_PENDING;
    return ORAS_OK;
  }
  auto jt = S->done.find(ticket);
  if (jt == S->done.end()) return ORAS_ERR_INVALID_ARG;
  *out = jt->second;
  return ORAS_OK;
}

const char* oras_server_error(oras_server* S, int64_t ticket) {
  if (!S) return "";
  std::lock_guard<std::mutex> lk(S->mu);
  if (ticket <= 0) return S->err.c_str();
  auto it = S->errors.find(ticket);
  return it == S->errors.end() ? "" : it->second.c_str();
}

int oras_server_stats(oras_server* S, oras_server_counters* out) {
  if (!S || !out) return ORAS_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(S->mu);
  *out = S->st;
  out->queued = (int32_t)(S->plan_q.size() + S->ready_q.size());
  return ORAS_OK;
}

void oras_server_destroy(oras_server* S) {
  if (!S) return;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
    for (auto* q : S->plan_q) finish_locked(S, q, ORAS_ERR_STATE, "server destroyed before the request was planned");
    for (auto* q : S->ready_q) {
      oras_destroy(q->h);
      q->h = nullptr;
      finish_locked(S, q, ORAS_ERR_STATE, "server destroyed before the request was admitted");
    }
    S->plan_q.clear();
    S->ready_q.clear();
  }
  S->cv.notify_all();
  for (auto& t : S->planners) t.join();  // a planner finishes the set-up it is running
  for (auto& t : S->workers) t.join();   // a worker finishes the request it is running
  for (auto& kv : S->live) {
    if (kv.second->h) oras_destroy(kv.second->h);
    delete kv.second;
  }
  delete S;
}

}  // extern "C"
