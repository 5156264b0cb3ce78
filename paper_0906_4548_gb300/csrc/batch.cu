// Batches of independent PM realisations (see dgp_batch_* in include/dgp.h).
//
// The realisations are grouped into classes: those of one mesh size and
// precision in the nonlinear mode with FP32 mesh data and n <= 128, at most
// kClassMax to a class.  A class shares one stream, and a step of the class
// launches each kernel stage once for all its members (the member on the
// grid's z or y index), with the relaxation iterations of the class replayed
// as one CUDA graph; members iterate in lockstep and each stops by its own
// rules.  Realisations that form no class step alone on a stream of their
// own.  Every class or lone realisation has one persistent host worker (its
// waits block on events), so the classes run concurrently on the GPU.
#include <condition_variable>
#include <mutex>
#include <thread>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/dgp.h"
#include "internal.h"

namespace {

struct Unit {
  std::vector<int> members;  // realisation indices
  cudaStream_t stream = nullptr;
  cudaEvent_t done_ev = nullptr;
};

}  // namespace

struct dgp_batch {
  int count = 0;
  int device = 0;
  std::vector<dgp_ctx*> ctx;
  std::vector<Unit> units;
  cudaEvent_t start_ev = nullptr;
  std::vector<std::thread> workers;
  std::mutex m;
  std::condition_variable cv_work, cv_done;
  unsigned long long generation = 0;
  int pending = 0;
  bool quit = false;
  // the posted job
  dgp_particles* parts = nullptr;
  const double* a = nullptr;
  const double* da = nullptr;
  dgp_solve_info* info = nullptr;
  std::vector<int> rc;  // per realisation
};

namespace {

bool class_eligible(const dgp_params& p) {
  return p.gravity == DGP_GRAVITY_NL && !p.local_only && !(p.a_nonlinear > 0.0) && p.precision != DGP_FP64 &&
         p.n <= 128;
}

// One step of a unit: the class step, or (a lone realisation, or a class step refused
// for a bad argument) each member's own pm_step.
void step_unit(dgp_batch* b, const Unit& u) {
  const int m = (int)u.members.size();
  if (m > 1) {
    dgp_ctx* cs[dgp::kClassMax];
    dgp_particles pp[dgp::kClassMax];
    double a[dgp::kClassMax], da[dgp::kClassMax];
    dgp_solve_info inf[dgp::kClassMax];
    for (int k = 0; k < m; ++k) {
      const int i = u.members[k];
      cs[k] = b->ctx[i];
      pp[k] = b->parts[i];
      a[k] = b->a[i];
      da[k] = b->da[i];
    }
    const int r = dgp::step_class(cs, m, pp, a, da, b->info ? inf : nullptr);
    if (r != DGP_E_INVALID) {
      for (int k = 0; k < m; ++k) {
        const int i = u.members[k];
        b->rc[i] = r;
        if (b->info) b->info[i] = inf[k];
      }
      return;
    }
  }
  for (int k = 0; k < m; ++k) {
    const int i = u.members[k];
    b->rc[i] = pm_step(b->ctx[i], &b->parts[i], b->a[i], b->da[i], b->info ? &b->info[i] : nullptr);
  }
}

void worker_main(dgp_batch* b, int w) {
  const bool dev_ok = cudaSetDevice(b->device) == cudaSuccess;
  unsigned long long seen = 0;
  const Unit& u = b->units[w];
  for (;;) {
    std::unique_lock<std::mutex> lk(b->m);
    b->cv_work.wait(lk, [&] { return b->quit || b->generation != seen; });
    if (b->quit) return;
    seen = b->generation;
    lk.unlock();
    if (dev_ok) {
      step_unit(b, u);
    } else {
      for (int i : u.members) b->rc[i] = DGP_E_CUDA;
    }
    const bool synced =
        cudaEventRecord(u.done_ev, u.stream) == cudaSuccess && cudaEventSynchronize(u.done_ev) == cudaSuccess;
    lk.lock();
    if (!synced)
      for (int i : u.members)
        if (b->rc[i] == DGP_OK) b->rc[i] = DGP_E_CUDA;
    if (--b->pending == 0) b->cv_done.notify_all();
  }
}

void destroy_batch(dgp_batch* b) {
  {
    std::lock_guard<std::mutex> lk(b->m);
    b->quit = true;
  }
  b->cv_work.notify_all();
  for (auto& t : b->workers)
    if (t.joinable()) t.join();
  for (dgp_ctx* c : b->ctx)
    if (c) dgp_destroy(c);
  for (Unit& u : b->units) {
    if (u.stream) cudaStreamDestroy(u.stream);
    if (u.done_ev) cudaEventDestroy(u.done_ev);
  }
  if (b->start_ev) cudaEventDestroy(b->start_ev);
  delete b;
}

}  // namespace

extern "C" {

int dgp_batch_create(dgp_batch** out, int count, const dgp_params* params, const dgp_cosmology* cosmo) {
  if (!out) return DGP_E_INVALID;
  *out = nullptr;
  if (count < 1 || !params || !cosmo) return DGP_E_INVALID;
  dgp_batch* b = new (std::nothrow) dgp_batch;
  if (!b) return DGP_E_NOMEM;
  b->count = count;
  b->ctx.assign(count, nullptr);
  // classes: realisations of one mesh size and precision, in order of appearance
  std::vector<int> unit_of(count, -1);
  for (int i = 0; i < count; ++i) {
    if (unit_of[i] >= 0) continue;
    Unit u;
    u.members.push_back(i);
    if (class_eligible(params[i]))
      for (int j = i + 1; j < count && (int)u.members.size() < dgp::kClassMax; ++j)
        if (unit_of[j] < 0 && class_eligible(params[j]) && params[j].n == params[i].n &&
            params[j].precision == params[i].precision) {
          u.members.push_back(j);
          unit_of[j] = (int)b->units.size();
        }
    unit_of[i] = (int)b->units.size();
    b->units.push_back(u);
  }
  int rc = DGP_OK;
  if (cudaGetDevice(&b->device) != cudaSuccess ||
      cudaEventCreateWithFlags(&b->start_ev, cudaEventDisableTiming) != cudaSuccess)
    rc = DGP_E_CUDA;
  for (Unit& u : b->units) {
    if (rc != DGP_OK) break;
    if (cudaStreamCreateWithFlags(&u.stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&u.done_ev, cudaEventBlockingSync | cudaEventDisableTiming) != cudaSuccess) {
      rc = DGP_E_CUDA;
      break;
    }
    for (int i : u.members) {
      rc = dgp_init(&b->ctx[i], &params[i], cosmo, u.stream);
      if (rc != DGP_OK) break;
      rc = dgp_set_blocking_sync(b->ctx[i], 1);
      if (rc != DGP_OK) break;
    }
  }
  if (rc != DGP_OK) {
    destroy_batch(b);
    return rc;
  }
  b->rc.assign(count, DGP_OK);
  for (size_t w = 0; w < b->units.size(); ++w) b->workers.emplace_back(worker_main, b, (int)w);
  *out = b;
  return DGP_OK;
}

int dgp_batch_context(dgp_batch* b, int i, dgp_ctx** out) {
  if (!b || !out || i < 0 || i >= b->count) return DGP_E_INVALID;
  *out = b->ctx[i];
  return DGP_OK;
}

int dgp_batch_step(dgp_batch* b, dgp_particles* parts, const double* a, const double* da, dgp_solve_info* info,
                   void* cuda_stream) {
  if (!b || !parts || !a || !da) return DGP_E_INVALID;
  if (cuda_stream) {
    if (cudaEventRecord(b->start_ev, (cudaStream_t)cuda_stream) != cudaSuccess) return DGP_E_CUDA;
    for (const Unit& u : b->units)
      if (cudaStreamWaitEvent(u.stream, b->start_ev, 0) != cudaSuccess) return DGP_E_CUDA;
  }
  std::unique_lock<std::mutex> lk(b->m);
  b->parts = parts;
  b->a = a;
  b->da = da;
  b->info = info;
  b->pending = (int)b->units.size();
  ++b->generation;
  b->cv_work.notify_all();
  b->cv_done.wait(lk, [&] { return b->pending == 0; });
  for (int r : b->rc)
    if (r != DGP_OK) return r;
  return DGP_OK;
}

int dgp_batch_classes(dgp_batch* b, int* class_of, int* nclasses) {
  if (!b || !class_of || !nclasses) return DGP_E_INVALID;
  for (size_t w = 0; w < b->units.size(); ++w)
    for (int i : b->units[w].members) class_of[i] = (int)w;
  *nclasses = (int)b->units.size();
  return DGP_OK;
}

int dgp_batch_set_plane_pass(dgp_batch* b, int on) {
  if (!b) return DGP_E_INVALID;
  for (dgp_ctx* c : b->ctx) dgp::set_plane_pass(c, on != 0);
  return DGP_OK;
}

void dgp_batch_destroy(dgp_batch* b) {
  if (b) destroy_batch(b);
}

}  // extern "C"
