// Batched solves and the request server of the C ABI (gdm_solve_batch, gdm_server_*).
//
// Independent problems are the paper's "unit tasks" (spin channels / k-points solved fully in
// parallel, Sec. 2.4).  Here they run as concurrent solves on one GPU: a pool of worker
// threads, each owning one handle and one CUDA stream, takes problems from a shared queue; the
// handles' kernels overlap on the device through their streams.  A worker's handle is reused
// for every problem that fits its capacity (gdm's handle keeps the capacity's leading
// dimension), so allocation happens only when a larger problem arrives.
//
// Server: requests are copied at submission, queued in arrival order and admitted by a device
// memory budget for the workers' handles; a request that arrives while others run starts as
// soon as a worker is free (continuous batching at request granularity).  Results go to the
// caller's output buffer; gdm_wait / gdm_poll return the status, energy, solve information and
// the submission-to-completion latency.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "../../include/gdm.h"
#include "gdm_internal.h"
#include "handle.h"

using namespace gdm;

namespace {

double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch())
      .count();
}

// Size class of a handle that serves problems up to n: multiples of 256 up to 2048, of 1024
// above (bounded waste, few reallocations).
int64_t size_class(int64_t n) {
  if (n <= 2048) return (n + 255) / 256 * 256;
  return (n + 1023) / 1024 * 1024;
}

gdm_status apply_settings(gdm_handle* h, gdm_precision prec) {
  return gdm_set_precision(h, prec);
}

// Solve one problem on handle *hp (created or grown as needed).  Inputs are read from the
// given pointers; P (if any) receives the result.
gdm_status solve_one(gdm_handle** hp, int device, gdm_precision prec, int64_t n, int64_t n_occ,
                     const double* H, int64_t ldh, const double* S, int64_t lds, gdm_mem mem,
                     double* P, int64_t ldp, gdm_mem p_mem, gdm_result* res) {
  gdm_status st;
  if (*hp == nullptr || (*hp)->n_cap < n) {
    if (*hp != nullptr) {
      gdm_finalize(*hp);
      *hp = nullptr;
    }
    const int64_t cap = size_class(n);
    st = gdm_init(hp, cap, cap / 2 > 0 ? cap / 2 : 1, device);
    if (st != GDM_OK) return st;
  }
  gdm_handle* h = *hp;
  st = handle_reconfigure(h, n, n_occ);
  if (st == GDM_OK) st = apply_settings(h, prec);
  if (st == GDM_OK) st = gdm_set_overlap(h, S, lds, mem);
  if (st == GDM_OK) st = gdm_set_hamiltonian(h, H, ldh, mem);
  gdm_info info;
  memset(&info, 0, sizeof(info));
  double e = 0.0;
  if (st == GDM_OK) st = gdm_solve_dm(h, P, ldp, p_mem, &e, &info);
  if (res != nullptr) {
    res->status = st;
    res->energy = e;
    res->info = info;
  }
  return st;
}

bool valid_problem(const gdm_problem& p) {
  return p.n_basis >= 1 && p.n_occ > 0 && p.n_occ < p.n_basis && p.H != nullptr &&
         p.S != nullptr && p.ldh >= p.n_basis && p.lds >= p.n_basis &&
         (p.P == nullptr || p.ldp >= p.n_basis);
}

}  // namespace

// ==========================================================================================
// batch
// ==========================================================================================
namespace gdm {
gdm_status batch_solve_grouped(const gdm_problem* pr, int count, gdm_result* res, int device,
                               std::vector<int>* resolve);
void batch_release();
}  // namespace gdm

namespace {
gdm_status solve_concurrent(const gdm_problem* problems, int count, gdm_result* results,
                            int device, int conc, gdm_precision prec);
}  // namespace

extern "C" gdm_status gdm_solve_batch(const gdm_problem* problems, int count, gdm_result* results,
                                      const gdm_batch_config* cfg) {
  if (count < 0 || (count > 0 && (problems == nullptr || results == nullptr))) return GDM_ERR_ARG;
  for (int i = 0; i < count; ++i)
    if (!valid_problem(problems[i])) return GDM_ERR_ARG;
  const int device = cfg ? cfg->device : 0;
  int conc = (cfg && cfg->concurrency > 0) ? cfg->concurrency : 4;
  const gdm_precision prec = cfg ? cfg->precision : GDM_PREC_MIXED;
  const int engine = cfg ? cfg->engine : GDM_BATCH_GROUPED;
  if (engine != GDM_BATCH_GROUPED && engine != GDM_BATCH_CONCURRENT) return GDM_ERR_ARG;
  if (count == 0) return GDM_OK;
  if (prec != GDM_PREC_MIXED || engine == GDM_BATCH_CONCURRENT)
    return solve_concurrent(problems, count, results, device, conc, prec);
  // lockstep grouped batch; problems that fail in the lockstep are solved again alone
  std::vector<int> resolve;
  gdm_status st = batch_solve_grouped(problems, count, results, device, &resolve);
  if (st != GDM_OK) return st;
  std::vector<gdm_problem> again;
  std::vector<int> where;
  for (int i = 0; i < count; ++i)
    if (resolve[i]) {
      again.push_back(problems[i]);
      where.push_back(i);
    }
  if (!again.empty()) {
    std::vector<gdm_result> r2(again.size());
    solve_concurrent(again.data(), static_cast<int>(again.size()), r2.data(), device, conc, prec);
    for (size_t k = 0; k < again.size(); ++k) {
      r2[k].latency_ms += results[where[k]].latency_ms;
      results[where[k]] = r2[k];
    }
  }
  for (int i = 0; i < count; ++i)
    if (results[i].status != GDM_OK && results[i].status != GDM_ERR_NOT_CONVERGED)
      return results[i].status;
  return GDM_OK;
}

extern "C" void gdm_batch_release(void) { batch_release(); }

namespace {
gdm_status solve_concurrent(const gdm_problem* problems, int count, gdm_result* results,
                            int device, int conc, gdm_precision prec) {
  if (conc > count) conc = count;
  // largest first, so each worker's first problem sizes its handle for the rest
  std::vector<int> order(count);
  for (int i = 0; i < count; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
    return problems[a].n_basis > problems[b].n_basis;
  });
  std::atomic<int> next{0};
  std::vector<std::thread> workers;
  for (int w = 0; w < conc; ++w) {
    workers.emplace_back([&]() {
      cudaSetDevice(device);
      gdm_handle* h = nullptr;
      for (;;) {
        const int k = next.fetch_add(1);
        if (k >= count) break;
        const gdm_problem& p = problems[order[k]];
        gdm_result* r = &results[order[k]];
        memset(r, 0, sizeof(*r));
        const double t0 = now_s();
        solve_one(&h, device, prec, p.n_basis, p.n_occ, p.H, p.ldh, p.S, p.lds, p.mem, p.P,
                  p.ldp, p.p_mem, r);
        r->latency_ms = (now_s() - t0) * 1e3;
      }
      if (h != nullptr) gdm_finalize(h);
    });
  }
  for (auto& t : workers) t.join();
  for (int i = 0; i < count; ++i)
    if (results[i].status != GDM_OK && results[i].status != GDM_ERR_NOT_CONVERGED)
      return results[i].status;
  return GDM_OK;
}
}  // namespace

// ==========================================================================================
// server
// ==========================================================================================
namespace {

struct Request {
  uint64_t ticket = 0;
  int64_t n = 0, n_occ = 0;
  std::vector<double> H, S;  // copies taken at submission (dense, ld = n)
  double* P = nullptr;
  int64_t ldp = 0;
  gdm_mem p_mem = GDM_MEM_HOST;
  double t_submit = 0.0;
  bool done = false;
  gdm_result result{};
};

}  // namespace

struct gdm_server {
  gdm_server_config cfg{};
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Request*> queue;
  std::map<uint64_t, Request*> requests;
  uint64_t next_ticket = 1;
  bool stopping = false;
  size_t in_use = 0;  // device bytes held by the workers' handles
  std::vector<std::thread> workers;
};

namespace {

void server_worker(gdm_server* s) {
  cudaSetDevice(s->cfg.device);
  gdm_handle* h = nullptr;
  size_t held = 0;
  for (;;) {
    Request* rq = nullptr;
    size_t need = 0;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      for (;;) {
        if (s->stopping) break;
        if (!s->queue.empty()) {
          Request* head = s->queue.front();
          const int64_t cap = size_class(head->n);
          need = (h != nullptr && h->n_cap >= head->n) ? held : handle_pool_bytes(cap);
          // admission: the handles of all workers must stay within the budget
          if (s->in_use - held + need <= s->cfg.hbm_budget_bytes) {
            rq = head;
            s->queue.pop_front();
            s->in_use = s->in_use - held + need;
            break;
          }
          if (h != nullptr && held > 0 && (h->n_cap < head->n)) {
            // this worker's handle is too small for the head anyway: give its memory back
            gdm_finalize(h);
            h = nullptr;
            s->in_use -= held;
            held = 0;
            continue;
          }
        }
        s->cv_work.wait_for(lk, std::chrono::milliseconds(50));
      }
      if (rq == nullptr) break;
    }
    if (h != nullptr && h->n_cap < rq->n) {
      gdm_finalize(h);
      h = nullptr;
    }
    held = need;
    solve_one(&h, s->cfg.device, s->cfg.precision, rq->n, rq->n_occ, rq->H.data(), rq->n,
              rq->S.data(), rq->n, GDM_MEM_HOST, rq->P, rq->ldp, rq->p_mem, &rq->result);
    if (h == nullptr) {  // allocation failed: nothing is held
      std::lock_guard<std::mutex> lk(s->mu);
      s->in_use -= held;
      held = 0;
    }
    {
      std::lock_guard<std::mutex> lk(s->mu);
      rq->result.latency_ms = (now_s() - rq->t_submit) * 1e3;
      rq->H.clear();
      rq->H.shrink_to_fit();
      rq->S.clear();
      rq->S.shrink_to_fit();
      rq->done = true;
    }
    s->cv_done.notify_all();
    s->cv_work.notify_all();
  }
  if (h != nullptr) gdm_finalize(h);
  std::lock_guard<std::mutex> lk(s->mu);
  s->in_use -= held;
}

gdm_status copy_in(std::vector<double>& dst, const double* src, int64_t n, int64_t ld,
                   gdm_mem mem) {
  dst.resize(static_cast<size_t>(n) * n);
  if (mem == GDM_MEM_HOST) {
    for (int64_t i = 0; i < n; ++i) memcpy(&dst[i * n], src + i * ld, sizeof(double) * n);
    return GDM_OK;
  }
  cudaError_t e = cudaMemcpy2D(dst.data(), sizeof(double) * n, src, sizeof(double) * ld,
                               sizeof(double) * n, n, cudaMemcpyDeviceToHost);
  return e == cudaSuccess ? GDM_OK : GDM_ERR_CUDA;
}

}  // namespace

extern "C" {

gdm_status gdm_server_create(gdm_server** out, const gdm_server_config* cfg) {
  if (out == nullptr) return GDM_ERR_ARG;
  *out = nullptr;
  gdm_server* s = new gdm_server();
  if (cfg != nullptr) s->cfg = *cfg;
  if (s->cfg.slots <= 0) s->cfg.slots = 4;
  if (s->cfg.slots > 64) s->cfg.slots = 64;
  if (s->cfg.hbm_budget_bytes == 0) s->cfg.hbm_budget_bytes = 120ull << 30;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || s->cfg.device < 0 || s->cfg.device >= ndev) {
    delete s;
    return GDM_ERR_ARG;
  }
  for (int i = 0; i < s->cfg.slots; ++i) s->workers.emplace_back(server_worker, s);
  *out = s;
  return GDM_OK;
}

gdm_status gdm_submit(gdm_server* s, const gdm_request* r, uint64_t* ticket) {
  if (s == nullptr || r == nullptr || ticket == nullptr) return GDM_ERR_ARG;
  if (r->n_basis < 1 || r->n_occ <= 0 || r->n_occ >= r->n_basis || r->H == nullptr ||
      r->S == nullptr || r->ldh < r->n_basis || r->lds < r->n_basis ||
      (r->P != nullptr && r->ldp < r->n_basis))
    return GDM_ERR_ARG;
  if (handle_pool_bytes(size_class(r->n_basis)) > s->cfg.hbm_budget_bytes) return GDM_ERR_BUDGET;
  Request* rq = new Request();
  rq->n = r->n_basis;
  rq->n_occ = r->n_occ;
  rq->P = r->P;
  rq->ldp = r->ldp;
  rq->p_mem = r->p_mem;
  gdm_status st = copy_in(rq->H, r->H, r->n_basis, r->ldh, r->mem);
  if (st == GDM_OK) st = copy_in(rq->S, r->S, r->n_basis, r->lds, r->mem);
  if (st != GDM_OK) {
    delete rq;
    return st;
  }
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stopping) {
      delete rq;
      return GDM_ERR_STATE;
    }
    rq->ticket = s->next_ticket++;
    rq->t_submit = now_s();
    s->requests[rq->ticket] = rq;
    s->queue.push_back(rq);
    *ticket = rq->ticket;
  }
  s->cv_work.notify_one();
  return GDM_OK;
}

gdm_status gdm_poll(gdm_server* s, uint64_t ticket, int* done, gdm_result* out) {
  if (s == nullptr || done == nullptr) return GDM_ERR_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->requests.find(ticket);
  if (it == s->requests.end()) return GDM_ERR_ARG;
  *done = it->second->done ? 1 : 0;
  if (!it->second->done) return GDM_OK;
  if (out != nullptr) *out = it->second->result;
  delete it->second;
  s->requests.erase(it);
  return GDM_OK;
}

gdm_status gdm_wait(gdm_server* s, uint64_t ticket, double timeout_s, gdm_result* out) {
  if (s == nullptr) return GDM_ERR_ARG;
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->requests.find(ticket);
  if (it == s->requests.end()) return GDM_ERR_ARG;
  Request* rq = it->second;
  const auto deadline = std::chrono::steady_clock::now() +
                        std::chrono::duration_cast<std::chrono::steady_clock::duration>(
                            std::chrono::duration<double>(timeout_s > 0 ? timeout_s : 0.0));
  while (!rq->done) {
    if (timeout_s >= 0 && std::chrono::steady_clock::now() >= deadline) return GDM_ERR_TIMEOUT;
    s->cv_done.wait_until(lk, timeout_s >= 0 ? deadline
                                             : std::chrono::steady_clock::now() +
                                                   std::chrono::milliseconds(100));
  }
  if (out != nullptr) *out = rq->result;
  delete rq;
  s->requests.erase(it);
  return GDM_OK;
}

gdm_status gdm_server_destroy(gdm_server* s) {
  if (s == nullptr) return GDM_OK;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stopping = true;
    for (Request* rq : s->queue) {  // never started: report them as cancelled
      rq->result.status = GDM_ERR_STATE;
      rq->done = true;
    }
    s->queue.clear();
  }
  s->cv_work.notify_all();
  for (auto& t : s->workers) t.join();
  for (auto& kv : s->requests) delete kv.second;
  s->requests.clear();
  delete s;
  return GDM_OK;
}

}  // extern "C"
