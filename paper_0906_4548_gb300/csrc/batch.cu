// Batches of independent PM realisations (see dgp_batch_* in include/dgp.h).
//
// Each realisation is a context with its own non-blocking stream and its own
// persistent host worker.  A step posts one job to all workers; each worker
// runs pm_step on its context (the relaxation's verdict waits block on an
// event, so waiting workers do not hold host cores) and finally waits for its
// stream, so the GPU sees the small kernels of all realisations at once.
#include <condition_variable>
#include <mutex>
#include <thread>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/dgp.h"

struct dgp_batch {
  int count = 0;
  int device = 0;
  std::vector<dgp_ctx*> ctx;
  std::vector<cudaStream_t> streams;
  std::vector<cudaEvent_t> done_ev;  // blocking-sync events, one per worker
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
  std::vector<int> rc;
};

namespace {

void worker_main(dgp_batch* b, int i) {
  const bool dev_ok = cudaSetDevice(b->device) == cudaSuccess;
  unsigned long long seen = 0;
  for (;;) {
    std::unique_lock<std::mutex> lk(b->m);
    b->cv_work.wait(lk, [&] { return b->quit || b->generation != seen; });
    if (b->quit) return;
    seen = b->generation;
    dgp_particles* pp = &b->parts[i];
    const double a = b->a[i], da = b->da[i];
    dgp_solve_info* inf = b->info ? &b->info[i] : nullptr;
    lk.unlock();
    int r = dev_ok ? pm_step(b->ctx[i], pp, a, da, inf) : DGP_E_CUDA;
    if (cudaEventRecord(b->done_ev[i], b->streams[i]) != cudaSuccess ||
        cudaEventSynchronize(b->done_ev[i]) != cudaSuccess)
      if (r == DGP_OK) r = DGP_E_CUDA;
    lk.lock();
    b->rc[i] = r;
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
  for (dgp_ctx* c : b->ctx) dgp_destroy(c);
  for (cudaStream_t s : b->streams) cudaStreamDestroy(s);
  for (cudaEvent_t e : b->done_ev) cudaEventDestroy(e);
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
  int rc = DGP_OK;
  if (cudaGetDevice(&b->device) != cudaSuccess ||
      cudaEventCreateWithFlags(&b->start_ev, cudaEventDisableTiming) != cudaSuccess)
    rc = DGP_E_CUDA;
  for (int i = 0; i < count && rc == DGP_OK; ++i) {
    cudaStream_t s = nullptr;
    cudaEvent_t e = nullptr;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) { rc = DGP_E_CUDA; break; }
    b->streams.push_back(s);
    if (cudaEventCreateWithFlags(&e, cudaEventBlockingSync | cudaEventDisableTiming) != cudaSuccess) {
      rc = DGP_E_CUDA;
      break;
    }
    b->done_ev.push_back(e);
    dgp_ctx* c = nullptr;
    rc = dgp_init(&c, &params[i], cosmo, s);
    if (rc != DGP_OK) break;
    b->ctx.push_back(c);
    rc = dgp_set_blocking_sync(c, 1);
  }
  if (rc != DGP_OK) {
    destroy_batch(b);
    return rc;
  }
  b->rc.assign(count, DGP_OK);
  for (int i = 0; i < count; ++i) b->workers.emplace_back(worker_main, b, i);
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
    for (cudaStream_t s : b->streams)
      if (cudaStreamWaitEvent(s, b->start_ev, 0) != cudaSuccess) return DGP_E_CUDA;
  }
  std::unique_lock<std::mutex> lk(b->m);
  b->parts = parts;
  b->a = a;
  b->da = da;
  b->info = info;
  b->pending = b->count;
  ++b->generation;
  b->cv_work.notify_all();
  b->cv_done.wait(lk, [&] { return b->pending == 0; });
  for (int r : b->rc)
    if (r != DGP_OK) return r;
  return DGP_OK;
}

void dgp_batch_destroy(dgp_batch* b) {
  if (b) destroy_batch(b);
}

}  // extern "C"
