// Serving: continuous batching of solve requests.
//
// A server owns a pool of worker threads.  Each worker has its own CUDA stream
// and runs one request at a time from start to end: the copy of the network
// and the right-hand sides to the device, the assembly of K, the operator, the
// preconditioner set-up and PCG for every right-hand side, and the copy of the
// solutions back.  Requests wait in a FIFO queue and are admitted when a worker
// is free and the device memory the request is estimated to need fits the
// budget (the free memory when the server was created, less a reserve, less
// the estimates of the requests running); a request whose estimate alone
// exceeds the budget is refused at submission.  The work of admitted requests
// overlaps on the GPU (different streams).  Nothing a request computes depends
// on what else runs: every kernel reduces in a fixed order, so a result is the
// same alone and in the mix.
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "spnet_internal.cuh"

using Clock = std::chrono::steady_clock;

namespace {

struct Job {
  spnet_request req;
  spnet_result res;
  Clock::time_point submit, admit;
  int64_t est = 0;
  bool done = false;
};

double ms_between(Clock::time_point a, Clock::time_point b) {
  return std::chrono::duration<double, std::milli>(b - a).count();
}

}  // namespace

struct spnet_server_s {
  int device = 0;
  int64_t budget = 0;     // bytes the running requests may hold
  int64_t committed = 0;  // estimates of the running requests
  int running = 0;
  bool stop = false;
  std::mutex mu;
  std::condition_variable cv_queue;  // a job was queued, or memory was released
  std::condition_variable cv_done;   // a job finished
  std::deque<int64_t> queue;
  std::map<int64_t, Job> jobs;
  int64_t next_ticket = 1;
  cudaEvent_t epoch = nullptr;  // device-time origin of the results' start/end stamps
  std::vector<std::thread> workers;
};

namespace spnet {

// device bytes a request is estimated to need at its peak (set-up): the
// operator and its copies of K, the preconditioner (star factors and solve
// windows, corner tables, the dense A_0 and its inverse tiles), PCG vectors
int64_t request_estimate(const spnet_request* r) {
  const int ndof = r->model == SPNET_MODEL_TRUSS3 ? 3 : 1;
  const int64_t n_dof = r->n_nodes * ndof;
  const int64_t nnz = (int64_t)ndof * ndof * (r->n_nodes + 2 * r->n_edges);
  int64_t m0 = ndof;
  for (int a = 0; a < r->dim; ++a) m0 *= (int64_t)(r->domain_hi[a] / r->H + 1.5);
  const int corners = 1 << r->dim;
  int64_t b = 48 * nnz + n_dof * (256 + 96 * (int64_t)corners) + 20 * m0 * m0;
  b += (int64_t)r->nrhs * n_dof * 24 + r->n_edges * 48 + (64ll << 20);
  // right-hand sides stepped together: five block vectors, the star results (about eight
  // entries per dof) and the coarse product's parts, for the block width
  const int64_t kb = r->nrhs < r->opts.batch_rhs ? r->nrhs : r->opts.batch_rhs;
  if (kb >= 2) b += kb * n_dof * (40 + 64) + 2 * m0 * m0 + kb * 16 * m0;
  return b;
}

static void run_job(spnet_server_s* sv, Job& job, cudaStream_t s, cudaEvent_t ev0, cudaEvent_t ev1) {
  const spnet_request& q = job.req;
  spnet_result& res = job.res;
  const int ndof = q.model == SPNET_MODEL_TRUSS3 ? 3 : 1;
  const int64_t n_dof = q.n_nodes * ndof;
  const int64_t cap = (int64_t)ndof * ndof * (q.n_nodes + 2 * q.n_edges);
  DevArena mem;
  mem.stream = s;
  struct Guard {
    DevArena& a;
    ~Guard() { a.free_all(); }
  } guard{mem};
  spnet_op_t op = nullptr;
  spnet_pc_t pc = nullptr;
  auto finish = [&](int rc) {
    if (pc) spnet_pc_destroy(pc);
    if (op) spnet_op_destroy(op);
    res.status = rc;
    if (rc != SPNET_OK) {
      std::strncpy(res.message, last_error().c_str(), sizeof(res.message) - 1);
      res.message[sizeof(res.message) - 1] = 0;
    }
  };
  int rc = SPNET_OK;
  int64_t *edges = nullptr, *dd = nullptr, *rp = nullptr;
  double *coef = nullptr, *dirs = nullptr, *coords = nullptr, *val = nullptr, *f = nullptr, *g = nullptr,
         *x = nullptr;
  int32_t* col = nullptr;
  cudaEventRecord(ev0, s);
  if ((rc = mem.get(&edges, 2 * q.n_edges + 1)) || (rc = mem.get(&coef, q.n_edges + 1)) ||
      (rc = mem.get(&coords, q.n_nodes * q.dim + 1)) || (rc = mem.get(&dd, q.n_dirichlet + 1)) ||
      (rc = mem.get(&rp, n_dof + 1)) || (rc = mem.get(&col, cap + 1)) || (rc = mem.get(&val, cap + 1)) ||
      (rc = mem.get(&f, (int64_t)q.nrhs * n_dof + 1)) || (rc = mem.get(&g, (int64_t)q.nrhs * q.n_dirichlet + 1)) ||
      (rc = mem.get(&x, (int64_t)q.nrhs * n_dof + 1)))
    return finish(rc);
  if (q.model == SPNET_MODEL_TRUSS3 && (rc = mem.get(&dirs, 3 * q.n_edges + 1))) return finish(rc);
  auto h2d = [&](void* d, const void* h, size_t bytes) {
    return bytes ? cudaMemcpyAsync(d, h, bytes, cudaMemcpyHostToDevice, s) : cudaSuccess;
  };
  if (h2d(edges, q.edges, sizeof(int64_t) * 2 * q.n_edges) || h2d(coef, q.coef, sizeof(double) * q.n_edges) ||
      h2d(coords, q.coords, sizeof(double) * q.n_nodes * q.dim) ||
      h2d(dd, q.dirichlet_dofs, sizeof(int64_t) * q.n_dirichlet) ||
      h2d(f, q.f, sizeof(double) * q.nrhs * n_dof) || h2d(g, q.g, sizeof(double) * q.nrhs * q.n_dirichlet) ||
      (dirs && h2d(dirs, q.dirs, sizeof(double) * 3 * q.n_edges)))
    return finish(fail(SPNET_ERR_CUDA, "serve: copy of the request to the device failed"));
  int64_t nnz = 0;
  if ((rc = spnet_assemble(q.model, q.n_nodes, q.n_edges, edges, coef, dirs, SPNET_MEM_DEVICE, s, rp, col, val,
                           cap, &nnz)))
    return finish(rc);
  if ((rc = build_network_operator(q.dim, ndof, q.n_nodes, coords, rp, col, val, q.n_dirichlet, dd, q.domain_hi,
                                   SPNET_MEM_DEVICE, s, &op)))
    return finish(rc);
  if ((rc = setup_preconditioner(op, q.H, q.gamma_faces, &q.opts, &pc))) return finish(rc);
  std::vector<spnet_stats> st(q.nrhs);
  rc = pcg_solve(op, pc, q.nrhs, f, g, x, 0, q.rtol, q.maxit, SPNET_MEM_DEVICE, st.data());
  if (rc != SPNET_OK && rc != SPNET_ERR_NO_CONVERGENCE) return finish(rc);
  const int solve_rc = rc;
  if (cudaMemcpyAsync(q.x, x, sizeof(double) * q.nrhs * n_dof, cudaMemcpyDeviceToHost, s) != cudaSuccess)
    return finish(fail(SPNET_ERR_CUDA, "serve: copy of the solution to the host failed"));
  cudaEventRecord(ev1, s);
  if (cudaStreamSynchronize(s) != cudaSuccess)
    return finish(fail(SPNET_ERR_CUDA, "serve: the request's stream failed"));
  res.iterations = 0;
  res.relres = 0.0;
  for (int k = 0; k < q.nrhs; ++k) {
    res.iterations = st[k].iterations > res.iterations ? st[k].iterations : res.iterations;
    res.relres = st[k].relres > res.relres ? st[k].relres : res.relres;
  }
  float t0 = 0.f, t1 = 0.f;
  cudaEventElapsedTime(&t0, sv->epoch, ev0);
  cudaEventElapsedTime(&t1, sv->epoch, ev1);
  res.device_start_ms = t0;
  res.device_end_ms = t1;
  finish(solve_rc);
}

static void worker_main(spnet_server_s* sv) {
  cudaSetDevice(sv->device);
  cudaStream_t s = nullptr;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  const bool ok = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) == cudaSuccess &&
                  cudaEventCreate(&ev0) == cudaSuccess && cudaEventCreate(&ev1) == cudaSuccess;
  for (;;) {
    Job* job = nullptr;
    {
      std::unique_lock<std::mutex> lk(sv->mu);
      for (;;) {
        if (sv->stop && sv->queue.empty()) break;
        if (!sv->queue.empty()) {
          Job& head = sv->jobs[sv->queue.front()];
          // FIFO admission: the head waits until its estimate fits (it fits once nothing
          // else runs: submission refuses estimates beyond the budget)
          if (sv->committed + head.est <= sv->budget) {
            sv->queue.pop_front();
            job = &head;
            sv->committed += job->est;
            sv->running += 1;
            job->admit = Clock::now();
            break;
          }
        }
        sv->cv_queue.wait(lk);
      }
    }
    if (!job) break;
    if (!ok) {
      job->res.status = SPNET_ERR_CUDA;
      std::strncpy(job->res.message, "serve: the worker could not create its stream", sizeof(job->res.message) - 1);
    } else {
      run_job(sv, *job, s, ev0, ev1);
    }
    const Clock::time_point end = Clock::now();
    {
      std::lock_guard<std::mutex> lk(sv->mu);
      job->res.queue_ms = ms_between(job->submit, job->admit);
      job->res.latency_ms = ms_between(job->submit, end);
      job->done = true;
      sv->committed -= job->est;
      sv->running -= 1;
    }
    sv->cv_done.notify_all();
    sv->cv_queue.notify_all();
  }
  if (ev0) cudaEventDestroy(ev0);
  if (ev1) cudaEventDestroy(ev1);
  if (s) cudaStreamDestroy(s);
}

}  // namespace spnet

using namespace spnet;

extern "C" int spnet_server_create(int max_inflight, int64_t reserve_bytes, spnet_server_t* out) {
  cudaGetLastError();  // start from a clean error state
  if (!out || max_inflight < 1 || max_inflight > 64 || reserve_bytes < 0)
    return fail(SPNET_ERR_BAD_INPUT, "spnet_server_create: max_inflight in 1..64, reserve_bytes >= 0");
  *out = nullptr;
  spnet_server_s* sv = new spnet_server_s();
  if (cudaGetDevice(&sv->device) != cudaSuccess) {
    delete sv;
    return fail(SPNET_ERR_CUDA, "spnet_server_create: no CUDA device");
  }
  size_t free_b = 0, total_b = 0;
  if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess || cudaEventCreate(&sv->epoch) != cudaSuccess) {
    delete sv;
    return fail(SPNET_ERR_CUDA, "spnet_server_create: device query failed");
  }
  cudaEventRecord(sv->epoch, 0);
  cudaEventSynchronize(sv->epoch);
  sv->budget = (int64_t)free_b - reserve_bytes;
  if (sv->budget <= 0) {
    cudaEventDestroy(sv->epoch);
    delete sv;
    return fail(SPNET_ERR_NO_MEMORY, "spnet_server_create: the reserve exceeds the free device memory");
  }
  for (int i = 0; i < max_inflight; ++i) sv->workers.emplace_back(worker_main, sv);
  *out = sv;
  return SPNET_OK;
}

extern "C" int spnet_server_submit(spnet_server_t sv, const spnet_request* req, int64_t* ticket) {
  cudaGetLastError();
  if (!sv || !req || !ticket) return fail(SPNET_ERR_BAD_INPUT, "spnet_server_submit: null argument");
  const spnet_request& q = *req;
  if ((q.model != SPNET_MODEL_SCALAR && q.model != SPNET_MODEL_TRUSS3) || (q.dim != 2 && q.dim != 3) ||
      q.n_nodes < 1 || q.n_edges < 0 || q.nrhs < 1 || q.n_dirichlet < 0 || !q.edges || !q.coef || !q.coords ||
      !q.f || !q.g || !q.x || (q.model == SPNET_MODEL_TRUSS3 && !q.dirs) || (q.n_dirichlet > 0 && !q.dirichlet_dofs) ||
      !(q.H > 0) || !(q.rtol > 0) || q.maxit < 1)
    return fail(SPNET_ERR_BAD_INPUT, "spnet_server_submit: malformed request");
  const int64_t est = request_estimate(&q);
  std::lock_guard<std::mutex> lk(sv->mu);
  if (sv->stop) return fail(SPNET_ERR_BAD_INPUT, "spnet_server_submit: the server is shutting down");
  if (est > sv->budget)
    return fail(SPNET_ERR_NO_MEMORY, "spnet_server_submit: the request is estimated to need " +
                                         std::to_string(est) + " device bytes, more than the server's budget of " +
                                         std::to_string(sv->budget));
  const int64_t t = sv->next_ticket++;
  Job& job = sv->jobs[t];
  job.req = q;
  job.res = spnet_result{};
  job.submit = Clock::now();
  job.est = est;
  sv->queue.push_back(t);
  *ticket = t;
  sv->cv_queue.notify_all();
  return SPNET_OK;
}

extern "C" int spnet_server_wait(spnet_server_t sv, int64_t ticket, spnet_result* out) {
  cudaGetLastError();
  if (!sv || !out) return fail(SPNET_ERR_BAD_INPUT, "spnet_server_wait: null argument");
  std::unique_lock<std::mutex> lk(sv->mu);
  auto it = sv->jobs.find(ticket);
  if (it == sv->jobs.end()) return fail(SPNET_ERR_BAD_INPUT, "spnet_server_wait: unknown ticket");
  sv->cv_done.wait(lk, [&] { return it->second.done; });
  *out = it->second.res;
  sv->jobs.erase(it);
  return SPNET_OK;
}

extern "C" int spnet_server_poll(spnet_server_t sv, int64_t ticket, spnet_result* out, int* done) {
  cudaGetLastError();
  if (!sv || !out || !done) return fail(SPNET_ERR_BAD_INPUT, "spnet_server_poll: null argument");
  std::lock_guard<std::mutex> lk(sv->mu);
  auto it = sv->jobs.find(ticket);
  if (it == sv->jobs.end()) return fail(SPNET_ERR_BAD_INPUT, "spnet_server_poll: unknown ticket");
  *done = it->second.done ? 1 : 0;
  if (*done) {
    *out = it->second.res;
    sv->jobs.erase(it);
  }
  return SPNET_OK;
}

extern "C" int spnet_server_cancel(spnet_server_t sv, int64_t ticket, int* cancelled) {
  cudaGetLastError();
  if (!sv || !cancelled) return fail(SPNET_ERR_BAD_INPUT, "spnet_server_cancel: null argument");
  *cancelled = 0;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    auto it = sv->jobs.find(ticket);
    if (it == sv->jobs.end()) return fail(SPNET_ERR_BAD_INPUT, "spnet_server_cancel: unknown ticket");
    for (auto q = sv->queue.begin(); q != sv->queue.end(); ++q) {
      if (*q != ticket) continue;
      sv->queue.erase(q);
      Job& job = it->second;
      job.res.status = SPNET_ERR_CANCELLED;
      std::strncpy(job.res.message, "cancelled before admission", sizeof(job.res.message) - 1);
      job.res.queue_ms = job.res.latency_ms = ms_between(job.submit, Clock::now());
      job.done = true;
      *cancelled = 1;
      break;
    }
  }
  if (*cancelled) {
    sv->cv_done.notify_all();
    sv->cv_queue.notify_all();  // the next request may now be the head
  }
  return SPNET_OK;
}

extern "C" int spnet_server_estimate(const spnet_request* req, int64_t* bytes) {
  if (!req || !bytes) return fail(SPNET_ERR_BAD_INPUT, "spnet_server_estimate: null argument");
  *bytes = request_estimate(req);
  return SPNET_OK;
}

extern "C" int spnet_server_budget(spnet_server_t sv, int64_t* bytes) {
  if (!sv || !bytes) return fail(SPNET_ERR_BAD_INPUT, "spnet_server_budget: null argument");
  std::lock_guard<std::mutex> lk(sv->mu);
  *bytes = sv->budget;
  return SPNET_OK;
}

extern "C" int spnet_server_destroy(spnet_server_t sv) {
  cudaGetLastError();
  if (!sv) return SPNET_OK;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->stop = true;
  }
  sv->cv_queue.notify_all();
  for (std::thread& w : sv->workers) w.join();
  if (sv->epoch) cudaEventDestroy(sv->epoch);
  delete sv;
  return SPNET_OK;
}
