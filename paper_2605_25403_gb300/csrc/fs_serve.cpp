// Continuous-batching request loop (no counterpart in the paper, whose
// workflow runs one simulation at a time; Sec. 3.1 ComputationModel).
//
// Requests (a structured mesh, a problem description and a number of time
// steps) wait in a FIFO queue.  A request is admitted when a slot is free and
// its estimated device footprint fits in the HBM budget left by the requests
// already resident.  Admitted requests are set up (mesh, device problem,
// multigrid hierarchies) by a pool of host threads while the GPU keeps
// working on the others, then stepped through the non-blocking step API on
// their own streams, so the kernels of all resident requests overlap on the
// device.  A finished request records its latency, optionally keeps its final
// state on the host, and releases its memory and slot for the next request.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "fs_internal.h"

struct fs_server {
  struct Req {
    int64_t id = 0;
    fs_mesh_desc mdesc{};
    fs_problem_desc pdesc{};
    int nsteps = 0;
    int keep_state = 0;
    double arrival = 0, admitted = 0, started = 0, finished = 0;
    int64_t est_bytes = 0, bytes = 0;
    fs_mesh* mesh = nullptr;
    fs_problem* prob = nullptr;
    std::atomic<int> setup_done{0};  // 1 ok, -1 failed (set by a worker)
    int setup_rc = FS_OK;
    int status = FS_OK;
    int iters = 0;
    std::vector<double> state;
  };

  fs_server_desc desc{};
  std::deque<std::shared_ptr<Req>> queue;  // waiting, FIFO
  std::vector<std::shared_ptr<Req>> setup, active;
  std::vector<fs_request_result> done;
  std::vector<std::shared_ptr<Req>> done_reqs;  // keep states until popped
  int64_t next_id = 1, bytes_reserved = 0;
  // set-up workers
  std::mutex mu;
  std::condition_variable cv;
  std::deque<std::shared_ptr<Req>> work;
  std::vector<std::thread> workers;
  bool stop = false;
  int device = 0;

  void worker() {
    cudaSetDevice(device);
    while (true) {
      std::shared_ptr<Req> r;
      {
        std::unique_lock<std::mutex> lk(mu);
        cv.wait(lk, [&] { return stop || !work.empty(); });
        if (stop && work.empty()) return;
        r = work.front();
        work.pop_front();
      }
      int rc = fs_mesh_create(&r->mdesc, &r->mesh);
      if (rc == FS_OK) rc = fs_problem_create(r->mesh, &r->pdesc, nullptr, &r->prob);
      r->setup_rc = rc;
      r->setup_done.store(rc == FS_OK ? 1 : -1);
    }
  }
};

namespace {

// Device footprint estimate of a request (bytes), from its sizes: mesh
// tables, FP64 blocks, vectors, the Krylov basis (m = 30) and the multigrid
// hierarchies (geometric series over the levels).
int64_t estimate_bytes(const fs_mesh_desc& md, int precision) {
  const int dim = md.dim;
  double cells = 1, n2 = 1, nv = 1;
  for (int a = 0; a < dim; ++a) {
    cells *= md.n[a];
    n2 *= 2.0 * md.n[a] + 1;
    nv *= md.n[a] + 1.0;
  }
  cells *= dim == 2 ? 2 : 6;
  const double nloc = dim == 2 ? 6 : 10, nb = dim + 1;
  const double ndof = dim * n2 + nv;
  const double nnzA = n2 * (dim == 2 ? 13.5 : 28.5), nnzB = nv * (dim == 2 ? 15 : 62);
  const double s = precision == FS_PREC_FP32_REFINE ? 4.0 : 8.0;
  double b = 0;
  b += cells * (4 * nloc + nloc * nloc + 2 * nb * nloc + nb * nb + 4);  // c2d, slots, colours
  b += n2 * (8 * dim + 1 + 4) + 4 * (2 * nnzA + 2 * nnzB) + 16 * (n2 + nv);  // geometry, patterns
  b += 8 * (3 * nnzA + 2 * dim * nnzB + nnzB + 3 * nv);              // FP64 values
  b += 8 * (4 * ndof + dim * n2);                                    // x, b, r, F
  b += 8.0 * fs::kExtrapMax * ndof;                                  // state history
  if (precision == FS_PREC_FP32_REFINE) b += 4 * (nnzA + 2 * dim * nnzB);
  b += s * (61.0 * ndof + dim * n2 + nv);                            // V, Z, work
  b += 1.6 * (s * nnzA + 4 * nnzA + 5 * s * dim * n2);              // hierarchies
  // dense coarsest inverses: large problems keep up to 3500 (3D) or 2000
  // (2D) rows per hierarchy, inverted on the device through an n x 2n FP64
  // workspace (one at a time, freed after set-up); smaller ones at most 800
  const bool big = n2 >= 100000;
  const double nc = big ? (dim == 3 ? 3500.0 : 2000.0) : 800.0;
  b += 2 * s * nc * nc + (big ? 16.0 * nc * nc : 0.0);
  // partial sums: tiles of up to 2048 entries, or up to four per SM when
  // the problem is small (counted for up to 256 SMs)
  b += 8.0 * 33 * std::max(ndof / 2048.0 + 2 * dim + 1, 1024.0);
  return (int64_t)(b * 1.1) + (64 << 20);
}

double finished_wall(fs_server::Req& r) { return r.finished; }

}  // namespace

extern "C" {

int fs_server_create(const fs_server_desc* desc, fs_server** out) {
  if (!desc || !out || desc->max_slots < 1 || desc->hbm_budget <= 0) {
    fs::set_error("fs_server_create: need max_slots >= 1 and a positive budget");
    return FS_ERR_INVALID_ARG;
  }
  auto* S = new (std::nothrow) fs_server;
  if (!S) return FS_ERR_OOM;
  S->desc = *desc;
  cudaGetDevice(&S->device);
  int nw = std::max(1, std::min(desc->setup_threads > 0 ? desc->setup_threads : 4, 16));
  for (int i = 0; i < nw; ++i) S->workers.emplace_back([S] { S->worker(); });
  *out = S;
  return FS_OK;
}

int fs_server_destroy(fs_server* S) {
  if (!S) return FS_OK;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
  }
  S->cv.notify_all();
  for (auto& t : S->workers) t.join();
  auto release = [](std::shared_ptr<fs_server::Req>& r) {
    if (r->prob) fs_problem_destroy(r->prob);
    if (r->mesh) fs_mesh_destroy(r->mesh);
    r->prob = nullptr;
    r->mesh = nullptr;
  };
  for (auto& r : S->setup) release(r);
  for (auto& r : S->active) release(r);
  delete S;
  return FS_OK;
}

int fs_server_submit(fs_server* S, const fs_mesh_desc* mdesc, const fs_problem_desc* pdesc,
                     int nsteps, double arrival, int keep_state, int64_t* id) {
  if (!S || !mdesc || !pdesc || nsteps < 1) {
    fs::set_error("fs_server_submit: bad argument");
    return FS_ERR_INVALID_ARG;
  }
  auto r = std::make_shared<fs_server::Req>();
  r->id = S->next_id++;
  r->mdesc = *mdesc;
  r->pdesc = *pdesc;
  r->nsteps = nsteps;
  r->keep_state = keep_state;
  r->arrival = arrival;
  r->est_bytes = estimate_bytes(*mdesc, pdesc->precision);
  if (r->est_bytes > S->desc.hbm_budget) {
    fs::set_error("fs_server_submit: the request's estimated footprint exceeds the budget");
    return FS_ERR_OOM;
  }
  S->queue.push_back(r);
  if (id) *id = r->id;
  return FS_OK;
}

int fs_server_progress(fs_server* S, double now, int* n_completed) {
  if (!S) {
    fs::set_error("fs_server_progress: null server");
    return FS_ERR_INVALID_ARG;
  }
  int completed = 0;
  // 1. admission (FIFO): a free slot and room in the budget
  while (!S->queue.empty()) {
    auto& head = S->queue.front();
    const int slots = (int)(S->setup.size() + S->active.size());
    if (slots >= S->desc.max_slots || S->bytes_reserved + head->est_bytes > S->desc.hbm_budget)
      break;
    head->admitted = now;
    S->bytes_reserved += head->est_bytes;
    {
      std::lock_guard<std::mutex> lk(S->mu);
      S->work.push_back(head);
    }
    S->cv.notify_one();
    S->setup.push_back(head);
    S->queue.pop_front();
  }
  auto finish = [&](std::shared_ptr<fs_server::Req>& r) {
    r->finished = now;
    if (r->prob) {
      if (r->keep_state) {
        fs_dofmap_info info;
        fs_dof_map(r->mesh, &info, nullptr, nullptr, nullptr, nullptr, nullptr);
        r->state.resize(info.n_dof);
        double t;
        fs_get_state(r->prob, r->state.data(), 1, &t);
      }
      fs_solve_stats st;
      if (fs_instance_stats(r->prob, &st) == FS_OK) r->iters = st.iters;
      fs_problem_destroy(r->prob);
      r->prob = nullptr;
    }
    if (r->mesh) fs_mesh_destroy(r->mesh);
    r->mesh = nullptr;
    S->bytes_reserved -= r->est_bytes;
    fs_request_result res{};
    res.id = r->id;
    res.status = r->status;
    res.arrival = r->arrival;
    res.admitted = r->admitted;
    res.started = r->started;
    res.finished = finished_wall(*r);
    res.nsteps = r->nsteps;
    res.iters = r->iters;
    res.device_bytes = r->bytes;
    S->done.push_back(res);
    if (r->keep_state) S->done_reqs.push_back(r);
    completed++;
  };
  // 2. set-up finished -> start stepping
  for (size_t i = 0; i < S->setup.size();) {
    auto r = S->setup[i];
    int st = r->setup_done.load();
    if (st == 0) {
      ++i;
      continue;
    }
    S->setup.erase(S->setup.begin() + i);
    if (st < 0) {
      r->status = r->setup_rc;
      finish(r);
      continue;
    }
    r->bytes = fs_problem_device_bytes(r->prob);
    if (r->bytes > r->est_bytes) {
      // an estimate that fell short: reserve what the problem really holds,
      // so later admissions see the budget that is actually left
      S->bytes_reserved += r->bytes - r->est_bytes;
      r->est_bytes = r->bytes;
    }
    r->started = now;
    int rc = fs_step_begin(r->prob, r->nsteps, nullptr);
    if (rc != FS_OK) {
      r->status = rc;
      finish(r);
      continue;
    }
    S->active.push_back(r);
  }
  // 3. advance every active request without blocking
  for (size_t i = 0; i < S->active.size();) {
    auto r = S->active[i];
    int isdone = 0;
    int rc = fs_step_poll(r->prob, 0, &isdone);
    if (isdone || rc != FS_OK) {
      r->status = rc;
      S->active.erase(S->active.begin() + i);
      finish(r);
      continue;
    }
    ++i;
  }
  if (n_completed) *n_completed = completed;
  return FS_OK;
}

int fs_server_pop_completed(fs_server* S, fs_request_result* out, int max, int* n) {
  if (!S || !n) {
    fs::set_error("fs_server_pop_completed: null argument");
    return FS_ERR_INVALID_ARG;
  }
  int k = std::min<int>(max, (int)S->done.size());
  if (out)
    for (int i = 0; i < k; ++i) out[i] = S->done[i];
  S->done.erase(S->done.begin(), S->done.begin() + k);
  *n = k;
  return FS_OK;
}

int fs_server_take_state(fs_server* S, int64_t id, double* x, int64_t n) {
  if (!S || !x) {
    fs::set_error("fs_server_take_state: null argument");
    return FS_ERR_INVALID_ARG;
  }
  for (size_t i = 0; i < S->done_reqs.size(); ++i) {
    auto& r = S->done_reqs[i];
    if (r->id != id) continue;
    if ((int64_t)r->state.size() != n) {
      fs::set_error("fs_server_take_state: size mismatch");
      return FS_ERR_INVALID_ARG;
    }
    std::memcpy(x, r->state.data(), sizeof(double) * n);
    S->done_reqs.erase(S->done_reqs.begin() + i);
    return FS_OK;
  }
  fs::set_error("fs_server_take_state: no kept state for this id");
  return FS_ERR_INVALID_ARG;
}

int fs_server_status(const fs_server* S, int* queued, int* resident, int64_t* bytes_reserved) {
  if (!S) {
    fs::set_error("fs_server_status: null server");
    return FS_ERR_INVALID_ARG;
  }
  if (queued) *queued = (int)S->queue.size();
  if (resident) *resident = (int)(S->setup.size() + S->active.size());
  if (bytes_reserved) *bytes_reserved = S->bytes_reserved;
  return FS_OK;
}

int64_t fs_server_estimate_bytes(const fs_mesh_desc* mdesc, int precision) {
  return mdesc ? estimate_bytes(*mdesc, precision) : 0;
}

}  // extern "C"
