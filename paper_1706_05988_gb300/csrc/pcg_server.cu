// Continuous-batching solve server (pcg_server_*, pcg_submit, pcg_poll).
//
// Requests are admitted into a device arena of fixed size (first fit); a request that
// does not fit waits on the host until earlier requests are polled and free their
// memory.  Admitted requests are published to a ring of work items in mapped host
// memory.  A persistent kernel of thread-block clusters takes items as clusters come
// free (compare-and-swap on a device counter), solves each one with the per-cluster
// solver of the batched launch, and raises the item's completion flag with a
// system-scope release.  Work that arrives while other requests run is taken by the
// next free cluster: requests overlap on the device.  With no published work for
// kIdleNs the kernel's clusters exit; the host relaunches the kernel when work arrives.
// Every wait of the kernel is bounded by %globaltimer.
//
// Requests of n >= kDeviceN take the whole GPU instead (the device lane): a preparing host
// thread creates their single-system solver contexts ahead, and two solving threads run
// pcg_solve on them, up to two at a time, while the cluster kernels are stopped.  Host
// passes over a request's arrays run on several threads (pcg_host_parallel.h).
#include <cuda/atomic>
#include <cuda_runtime.h>
#include <math.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <atomic>
#include <cstring>
#include <new>
#include <thread>
#include <vector>

#define PCG_KERNELS_IMPL
#include "../../include/pcg.h"

#include "pcg_host_parallel.h"
#include "pcg_server_kernel.cuh"

using namespace pcgk::srv;

using namespace pcgk;

namespace {

struct Request {
  uint64_t ticket;
  pcg_matrix A;                     // layout and dimensions (array pointers: see src below)
  // The request's arrays.  At submission they point at the caller's arrays; a request
  // that cannot be admitted at once copies them into the vectors below and points there.
  const double* b_src = nullptr;
  const int32_t *row_ptr_src = nullptr, *col_src = nullptr;
  const double *val_src = nullptr, *diag_src = nullptr, *ax_src = nullptr, *ay_src = nullptr, *az_src = nullptr;
  host::buffer<double> b;
  host::buffer<int32_t> row_ptr, col;
  host::buffer<double> val, diag, ax, ay, az;
  double tol, sigma;
  int method, maxit, family;
  int mode;                         // 0 binary64, 1 + Jacobi, 2 mixed, 3 mixed + Jacobi
  long long n, nnz;
  size_t bytes;                     // arena bytes
  size_t arena_off = 0;
  long long ring = -1;              // work-item index (in its lane's ring) once published
  int lane = 0;
  WorkItem item;                    // filled at admission, published when its copies are done
  uint32_t flags = 0;
  int precision = PCG_FP64;
  // device lane: the whole GPU, the single-system solver, a host worker thread
  bool device = false, device_done = false;
  pcg_ctx* ctx = nullptr;           // created ahead of the solve by the preparing thread
  pcg_status prep_status = PCG_OK;
  std::vector<double> x_host;
  std::vector<double> alpha_log, beta_log;   // device lane: alpha_i, beta_i of the solve
  pcg_result device_res{};
  pcg_status device_status = PCG_OK;
  cudaEvent_t uploaded = nullptr;   // staged admission: the copies' completion
  size_t stage_off = 0, stage_end = 0;
};

// One chunk of rows of a request's validation pass.
struct RowPass {
  double diag_sum = 0.0;   // sum of the rows' diagonals, left to right
  bool diag_ok = true;     // every diagonal positive and finite
  bool bad = false;        // a row_ptr range or a column index out of range
};

// Keeps the request's own copies of its arrays (it waits for memory; the caller's may go).
void own_arrays(Request* R) {
  const long long n = R->n;
  if (R->b.empty()) host::assign(R->b, R->b_src, (size_t)n);
  R->b_src = R->b.data();
  if (R->family == 4) {
    host::assign(R->row_ptr, R->row_ptr_src, (size_t)n + 1);
    host::assign(R->col, R->col_src, (size_t)R->nnz);
    host::assign(R->val, R->val_src, (size_t)R->nnz);
    R->row_ptr_src = R->row_ptr.data();
    R->col_src = R->col.data();
    R->val_src = R->val.data();
  } else if (R->family == 1 || R->family == 3) {
    host::assign(R->diag, R->diag_src, (size_t)n);
    host::assign(R->ax, R->ax_src, (size_t)n);
    host::assign(R->ay, R->ay_src, (size_t)n);
    R->diag_src = R->diag.data();
    R->ax_src = R->ax.data();
    R->ay_src = R->ay.data();
    if (R->family == 3) {
      host::assign(R->az, R->az_src, (size_t)n);
      R->az_src = R->az.data();
    }
  }
}

void release_arrays(Request* R) {
  R->b_src = nullptr;
  R->row_ptr_src = R->col_src = nullptr;
  R->val_src = R->diag_src = R->ax_src = R->ay_src = R->az_src = nullptr;
  host::buffer<int32_t>().swap(R->row_ptr);
  host::buffer<int32_t>().swap(R->col);
  for (host::buffer<double>* v : {&R->b, &R->val, &R->diag, &R->ax, &R->ay, &R->az}) host::buffer<double>().swap(*v);
}

}  // namespace

namespace {

// A lane is one persistent server kernel with its own cluster size, work ring and stream.
// Small requests go to a lane of many small clusters, large ones to a lane of few large
// clusters (a large request on a small cluster would set the tail latency); the two
// kernels run side by side on a fixed split of the GPU's resident blocks.
constexpr int kLanes = 2;
constexpr long long kLargeN = 32768;           // n at and above: the large lane
constexpr int kLaneCluster[kLanes] = {2, 16};
constexpr int kLargeLaneClusters = 8;         // clusters of the large lane (16 blocks each; measured
                                               // against 16 clusters of 8 on the 48-request trace:
                                               // span 1.84-1.85 s against 1.93-1.98 s)
// n at and above: the device lane.  Such a request needs the whole GPU's bandwidth, which
// no cluster has: the lanes finish their current requests and exit, the request runs on
// the single-system solver, and the lanes are relaunched.
constexpr long long kDeviceN = 1LL << 19;
// Smaller requests go first: a device request waits while the lanes hold published work
// that no cluster has claimed yet, but at most this long (so that a steady stream of small
// requests cannot hold it back).
constexpr auto kDeviceDefer = std::chrono::milliseconds(100);
constexpr int kDeviceSolvers = 2;   // whole-GPU solves that may run at the same time
constexpr int kPrepAhead = 3;       // device-lane contexts created and not yet destroyed

struct Lane {
  int csize = 2, clusters = 0;
  bool wide = false;                // the large lane's kernel has wide binary32 sweeps
  ServerShared* sh = nullptr;       // mapped host
  ServerShared* d_sh = nullptr;
  WorkItem* items = nullptr;        // mapped host
  WorkItem* d_items = nullptr;
  unsigned* done = nullptr;         // mapped host
  unsigned* d_done = nullptr;
  BatchOut* results = nullptr;      // mapped host
  BatchOut* d_results = nullptr;
  unsigned* d_claim = nullptr;      // device: items taken
  unsigned* d_left = nullptr;       // device: clusters still running
  std::vector<char> occupied;       // ring slot holds an item that was not polled yet
  cudaStream_t kstream = nullptr;
  unsigned published = 0;
};

}  // namespace

struct pcg_server {
  std::mutex mu;
  int device = 0;
  size_t budget = 0;
  int max_slots = 0;
  unsigned cap = 0;                 // ring capacity (per lane)
  char* arena = nullptr;            // device
  std::map<size_t, size_t> free_blocks;   // offset -> size (first fit, coalesced)
  Lane lane[kLanes];
  cudaStream_t cstream = nullptr;   // copies
  // device lane: `prep` creates the requests' solver contexts (validation, device memory,
  // the operator's upload) in order, at most kPrepAhead ahead of `worker`, which solves
  // them; so the uploads of the next requests overlap the current solve
  std::thread worker[kDeviceSolvers], prep;
  std::condition_variable cv, prep_cv;
  std::deque<Request*> prep_queue;              // submitted, context not yet created
  std::deque<Request*> device_queue;            // context created (or failed), not yet solved
  int prepared = 0;                             // contexts created and not yet destroyed
  bool quit = false;
  int device_active = 0;                        // whole-GPU solves running (the lanes stay down)
  pcg_status worker_error = PCG_OK;
  uint64_t next_ticket = 1;
  std::deque<Request*> waiting;                 // not yet admitted
  std::deque<Request*> uploading;               // admitted, copies in flight, not yet published
  std::map<uint64_t, Request*> inflight;        // admitted, not yet polled
  std::map<uint64_t, Request*> all;
  // pinned staging ring for admissions (one DMA per array instead of pageable copies
  // and a synchronisation per request); requests larger than the ring go the slow way
  char* stage = nullptr;
  size_t stage_cap = 0, stage_head = 0, stage_tail = 0;
  std::vector<cudaEvent_t> free_events;
};

namespace {

bool arena_alloc(pcg_server* S, size_t bytes, size_t* off) {
  for (auto it = S->free_blocks.begin(); it != S->free_blocks.end(); ++it) {
    if (it->second >= bytes) {
      *off = it->first;
      const size_t rest = it->second - bytes;
      const size_t o = it->first + bytes;
      S->free_blocks.erase(it);
      if (rest) S->free_blocks[o] = rest;
      return true;
    }
  }
  return false;
}

void arena_free(pcg_server* S, size_t off, size_t bytes) {
  auto it = S->free_blocks.emplace(off, bytes).first;
  auto nx = std::next(it);
  if (nx != S->free_blocks.end() && it->first + it->second == nx->first) {
    it->second += nx->second;
    S->free_blocks.erase(nx);
  }
  if (it != S->free_blocks.begin()) {
    auto pv = std::prev(it);
    if (pv->first + pv->second == it->first) {
      pv->second += it->second;
      S->free_blocks.erase(it);
    }
  }
}

size_t pad256(size_t b) { return (b + 255) & ~(size_t)255; }

// The request's alpha_i, beta_i log (i < kScalarLog) at the end of its arena block.
constexpr size_t kLogBytes = (2 * kScalarLog * sizeof(double) + 255) & ~(size_t)255;

size_t request_bytes(const Request& R) {
  const size_t n = (size_t)R.n, npad = (n + 31) & ~(size_t)31;
  const bool jac = R.mode & 1, mixed = R.mode >= 2;
  size_t b = (jac ? 16 : 8) * npad * sizeof(double);   // b, x, r, w0, w1, z, s, p (+ Jacobi vectors)
  if (R.family == 4) b += pad256((n + 1) * 4) + pad256(R.nnz * 4) + pad256(R.nnz * 8) + (mixed ? pad256(R.nnz * 4) : 0);
  if (R.family == 1 || R.family == 3) b += 4 * pad256(n * 8) + (mixed ? 4 * pad256(n * 4) : 0);
  return b + kLogBytes;
}

int family_of(const pcg_matrix& A) {
  if (A.layout == PCG_CSR32) return 4;
  if (A.layout == PCG_STENCIL5_2D) return A.diag ? 1 : 0;
  if (A.layout == PCG_STENCIL7_3D) return A.diag ? 3 : 2;
  return -1;
}

// Stage allocation in the pinned ring (FIFO: copies complete in submission order).
bool stage_alloc(pcg_server* S, size_t sz, size_t* off) {
  if (S->uploading.empty()) S->stage_head = S->stage_tail = 0;
  size_t& h = S->stage_head;
  const size_t t = S->stage_tail;
  if (h >= t) {
    if (S->stage_cap - h >= sz) {
      *off = h;
      h += sz;
      return true;
    }
    if (t > sz) {              // wrap to the front (strictly below the tail: head == tail means empty)
      *off = 0;
      h = sz;
      return true;
    }
    return false;
  }
  if (t - h > sz) {
    *off = h;
    h += sz;
    return true;
  }
  return false;
}

// Host bytes of an admission: b, then the binary64 operator arrays laid out as on the device.
size_t op64_bytes(const Request& R) {
  const size_t n = (size_t)R.n;
  if (R.family == 4) return pad256((n + 1) * 4) + pad256(R.nnz * 4) + pad256(R.nnz * 8);
  if (R.family == 1 || R.family == 3) return (R.family == 3 ? 4 : 3) * pad256(n * 8);
  return 0;
}

size_t stage_bytes(const Request& R) { return pad256((size_t)R.n * 8) + op64_bytes(R); }

// Places the request's data in its arena block and fills its work item.  With `staged`,
// b and the binary64 operator arrays are packed into the pinned ring at R->stage_off and
// copied with one DMA each, and R->uploaded marks the completion of the copies; otherwise the copies come straight from the request's arrays
// and are waited for here.  The binary32 copies and D^{-1} are derived on the device by the
// cluster that solves the request.
pcg_status upload(pcg_server* S, Request* R, bool staged) {
  char* base = S->arena + R->arena_off;
  const size_t n = (size_t)R->n, npad = (n + 31) & ~(size_t)31;
  const bool jac = R->mode & 1, mixed = R->mode >= 2;
  double* v = (double*)base;
  const size_t at0 = (jac ? 16 : 8) * npad * sizeof(double);
  size_t at = at0;
  char* hs = staged ? S->stage + R->stage_off : nullptr;   // host staging: [b | operator arrays]
  const size_t h_op = pad256(n * 8);
  auto put = [&](const void* src, size_t bytes) -> void* {
    if (at + pad256(bytes) > R->bytes) return nullptr;   // never: the layout is request_bytes'
    void* dst = base + at;
    if (staged) {
      host::copy(hs + h_op + (at - at0), src, bytes);
    } else if (bytes && cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, S->cstream) != cudaSuccess) {
      return nullptr;
    }
    at += pad256(bytes);
    return dst;
  };
  auto reserve32 = [&](size_t count) -> const float* {   // filled on the device by prepare_item
    if (at + pad256(count * 4) > R->bytes) return nullptr;
    void* dst = base + at;
    at += pad256(count * 4);
    return (const float*)dst;
  };
  BatchSys d{};
  d.layout = R->A.layout;
  d.n = (int)R->n;
  d.off = 0;
  d.log = (double*)(base + R->bytes - kLogBytes);
  d.sigma = R->method == PCG_SPCG ? R->sigma : 0.0;
  if (R->family == 4) {
    d.row_ptr = (const int*)put(R->row_ptr_src, (n + 1) * 4);
    d.col = (const int*)put(R->col_src, R->nnz * 4);
    d.val = (const double*)put(R->val_src, R->nnz * 8);
    if (!d.row_ptr || !d.col || !d.val) return PCG_ECUDA;
    if (mixed && !(d.val32 = reserve32(R->nnz))) return PCG_ECUDA;
  } else {
    d.nx = (int)R->A.nx;
    d.ny = (int)R->A.ny;
    d.nz = R->A.layout == PCG_STENCIL7_3D ? (int)R->A.nz : 1;
    if (R->family == 1 || R->family == 3) {
      d.diag = (const double*)put(R->diag_src, n * 8);
      d.ax = (const double*)put(R->ax_src, n * 8);
      d.ay = (const double*)put(R->ay_src, n * 8);
      d.az = R->family == 3 ? (const double*)put(R->az_src, n * 8) : nullptr;
      if (!d.diag || !d.ax || !d.ay || (R->family == 3 && !d.az)) return PCG_ECUDA;
      if (mixed) {
        d.diag32 = reserve32(n);
        d.ax32 = reserve32(n);
        d.ay32 = reserve32(n);
        d.az32 = R->family == 3 ? reserve32(n) : nullptr;
        if (!d.diag32 || !d.ax32 || !d.ay32 || (R->family == 3 && !d.az32)) return PCG_ECUDA;
      }
    }
  }
  const size_t op64 = op64_bytes(*R);
  if (staged) {
    host::copy(hs, R->b_src, n * 8);
    if (cudaMemcpyAsync(v, hs, n * 8, cudaMemcpyHostToDevice, S->cstream) != cudaSuccess) return PCG_ECUDA;
    if (op64 && cudaMemcpyAsync(base + at0, hs + h_op, op64, cudaMemcpyHostToDevice, S->cstream) != cudaSuccess)
      return PCG_ECUDA;
  } else if (cudaMemcpyAsync(v, R->b_src, n * 8, cudaMemcpyHostToDevice, S->cstream) != cudaSuccess) {
    return PCG_ECUDA;
  }
  if (staged) {
    if (cudaEventRecord(R->uploaded, S->cstream) != cudaSuccess) return PCG_ECUDA;
  } else if (cudaStreamSynchronize(S->cstream) != cudaSuccess) {
    return PCG_ECUDA;
  }
  WorkItem* w = &R->item;
  w->family = R->family;
  w->maxit = R->maxit;
  w->mode = R->mode;
  w->max_restarts = 200;
  w->eta = pcgk::kClusterMixedEta;
  w->tol = R->tol;
  w->sys = d;
  w->vec.stride = npad;
  w->vec.b = v;
  w->vec.x = v + npad;
  w->vec.r = v + 2 * npad;
  w->vec.w0 = v + 3 * npad;
  w->vec.w1 = v + 4 * npad;
  w->vec.z = v + 5 * npad;
  w->vec.s = v + 6 * npad;
  w->vec.p = v + 7 * npad;
  w->vec.u = w->vec.q = w->vec.t = w->vec.m0 = w->vec.m1 = w->vec.u64 = nullptr;
  w->vec.dinv = w->vec.dinv32 = nullptr;
  if (jac) {
    w->vec.u = v + 8 * npad;
    w->vec.q = v + 9 * npad;
    w->vec.t = v + 10 * npad;
    w->vec.m0 = v + 11 * npad;
    w->vec.m1 = v + 12 * npad;
    w->vec.u64 = v + 13 * npad;
    w->vec.dinv = v + 14 * npad;
    w->vec.dinv32 = v + 15 * npad;
  }
  return PCG_OK;
}

pcg_status launch_lane(pcg_server* S, Lane& L) {
  const unsigned left = (unsigned)L.clusters;
  if (cudaMemcpyAsync(L.d_left, &left, sizeof(unsigned), cudaMemcpyHostToDevice, L.kstream) != cudaSuccess)
    return PCG_ECUDA;
  if (cudaStreamSynchronize(L.kstream) != cudaSuccess) return PCG_ECUDA;
  L.sh->stop = 0;
  cuda::atomic_ref<unsigned, cuda::thread_scope_system> live(L.sh->live);
  live.store(1u, cuda::memory_order_release);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(L.clusters * L.csize);
  cfg.blockDim = dim3(kBlock);
  cfg.stream = L.kstream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = L.csize;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  const cudaError_t e = L.wide ? launch_server_wide(cfg, L.d_sh, L.d_items, L.d_results, L.d_done, S->cap, L.d_claim,
                                                   L.d_left)
                               : launch_server_t<false>(cfg, L.d_sh, L.d_items, L.d_results, L.d_done, S->cap,
                                                        L.d_claim, L.d_left);
  if (e != cudaSuccess) {
    cudaGetLastError();
    live.store(0u, cuda::memory_order_release);
    return PCG_ECUDA;
  }
  return PCG_OK;
}

// Publishes a request whose copies are done: its work item goes to the next ring slot.
void publish(pcg_server* S, Request* R) {
  Lane& L = S->lane[R->lane];
  const unsigned idx = L.published;
  L.items[idx % S->cap] = R->item;
  L.done[idx % S->cap] = 0;
  L.occupied[idx % S->cap] = 1;
  R->ring = idx;
  std::atomic_thread_fence(std::memory_order_seq_cst);
  cuda::atomic_ref<unsigned, cuda::thread_scope_system> tail(L.sh->tail);
  tail.store(idx + 1, cuda::memory_order_release);
  L.published = idx + 1;
}

bool slot_busy(const pcg_server* S, const Request* R) {
  const Lane& L = S->lane[R->lane];
  return L.occupied[L.published % S->cap] != 0;
}

// Publishes staged requests whose copies have completed (in order), admits waiting
// requests (FIFO) while arena memory, slots and staging allow, and makes sure a kernel
// runs while published work is unclaimed.
pcg_status pump(pcg_server* S) {
  for (;;) {
    while (!S->uploading.empty()) {
      Request* R = S->uploading.front();
      if (slot_busy(S, R)) break;                      // its ring slot still holds an unpolled request
      const cudaError_t q = cudaEventQuery(R->uploaded);
      if (q == cudaErrorNotReady) break;
      if (q != cudaSuccess) return PCG_ECUDA;
      publish(S, R);
      S->stage_tail = R->stage_end;
      S->free_events.push_back(R->uploaded);
      R->uploaded = nullptr;
      S->uploading.pop_front();
      if (S->uploading.empty()) S->stage_head = S->stage_tail = 0;
    }
    if (S->waiting.empty()) break;
    Request* R = S->waiting.front();
    if ((int)S->inflight.size() >= S->max_slots) break;
    const size_t sb = stage_bytes(*R);
    const bool staged = sb <= S->stage_cap;
    size_t soff = 0;
    const size_t head0 = S->stage_head, tail0 = S->stage_tail;
    if (staged && !stage_alloc(S, sb, &soff)) break;   // the ring drains as copies complete
    if (!staged && (!S->uploading.empty() || slot_busy(S, R))) break;
    size_t off;
    if (!arena_alloc(S, R->bytes, &off)) {
      S->stage_head = head0;                           // give the staging back
      S->stage_tail = tail0;
      break;
    }
    R->arena_off = off;
    if (staged) {
      if (S->free_events.empty()) {
        cudaEvent_t e;
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
          arena_free(S, off, R->bytes);
          S->stage_head = head0;
          S->stage_tail = tail0;
          return PCG_ECUDA;
        }
        S->free_events.push_back(e);
      }
      R->uploaded = S->free_events.back();
      S->free_events.pop_back();
      R->stage_off = soff;
      R->stage_end = soff + sb;
    }
    pcg_status s = upload(S, R, staged);
    if (s != PCG_OK) {
      arena_free(S, off, R->bytes);
      if (staged) {
        S->stage_head = head0;
        S->stage_tail = tail0;
        S->free_events.push_back(R->uploaded);
        R->uploaded = nullptr;
      }
      return s;
    }
    S->waiting.pop_front();
    S->inflight[R->ticket] = R;
    release_arrays(R);                 // the data is staged or on the device
    if (staged) {
      S->uploading.push_back(R);
    } else {
      publish(S, R);
    }
  }
  if (S->device_active > 0) return PCG_OK;   // the lanes stay down while a whole-GPU solve runs
  for (Lane& L : S->lane) {
    cuda::atomic_ref<unsigned, cuda::thread_scope_system> live(L.sh->live);
    cuda::atomic_ref<unsigned, cuda::thread_scope_system> claimed(L.sh->claimed);
    if (L.published > claimed.load(cuda::memory_order_acquire) && live.load(cuda::memory_order_acquire) == 0) {
      // the lane's previous kernel (if any) has exited: wait for its stream, then relaunch
      if (cudaStreamSynchronize(L.kstream) != cudaSuccess) return PCG_ECUDA;
      const pcg_status s = launch_lane(S, L);
      if (s != PCG_OK) return s;
    }
  }
  return PCG_OK;
}

// True while a lane has published work that no cluster has claimed.  (Requests whose
// copies are in flight do not count: one may wait for its ring slot, which only the
// caller's poll of an earlier request frees.)
bool lanes_pending(const pcg_server* S) {
  for (const Lane& L : S->lane) {
    cuda::atomic_ref<unsigned, cuda::thread_scope_system> claimed(L.sh->claimed);
    if (L.published > claimed.load(cuda::memory_order_acquire)) return true;
  }
  return false;
}

// The device lane's preparing thread: creates each request's solver context while the
// lanes and the previous device-lane solve run, then hands the request to the worker.
void prep_worker(pcg_server* S) {
  cudaSetDevice(S->device);
  std::unique_lock<std::mutex> lk(S->mu);
  for (;;) {
    S->prep_cv.wait(lk, [&] { return S->quit || (!S->prep_queue.empty() && S->prepared < kPrepAhead); });
    if (S->quit) return;
    Request* R = S->prep_queue.front();
    S->prep_queue.pop_front();
    ++S->prepared;
    lk.unlock();
    pcg_matrix A = R->A;
    A.row_ptr = R->row_ptr.empty() ? nullptr : R->row_ptr.data();
    A.col = R->col.empty() ? nullptr : R->col.data();
    A.val = R->val.empty() ? nullptr : R->val.data();
    A.diag = R->diag.empty() ? nullptr : R->diag.data();
    A.ax = R->ax.empty() ? nullptr : R->ax.data();
    A.ay = R->ay.empty() ? nullptr : R->ay.data();
    A.az = R->az.empty() ? nullptr : R->az.data();
    pcg_ctx* c = nullptr;
    R->prep_status = pcg_create(&A, R->flags, &c);
    R->ctx = c;
    // the operator is on the device now; b stays for pcg_solve
    host::buffer<int32_t>().swap(R->row_ptr);
    host::buffer<int32_t>().swap(R->col);
    for (host::buffer<double>* v : {&R->val, &R->diag, &R->ax, &R->ay, &R->az}) host::buffer<double>().swap(*v);
    R->x_host.assign((size_t)R->n, 0.0);
    R->alpha_log.assign((size_t)R->maxit + 1, NAN);
    R->beta_log.assign((size_t)R->maxit + 1, NAN);
    lk.lock();
    S->device_queue.push_back(R);
    S->cv.notify_all();
  }
}

// The device lane's solving threads (kDeviceSolvers of them): each takes the next prepared
// request and solves it with the single-system solver on the whole GPU, beside the other
// thread's solve (two mid-size solves together use the GPU better than one after the
// other).  The lanes stay down while any such solve runs.  Smaller requests first: when
// the lanes hold published work that no cluster has claimed, a thread waits until no
// whole-GPU solve runs, lets pump() relaunch the lanes and gives them up to kDeviceDefer to
// claim it; then it stops the lanes (their clusters finish what they hold and exit; every
// wait of theirs is bounded).
void device_worker(pcg_server* S) {
  cudaSetDevice(S->device);
  std::unique_lock<std::mutex> lk(S->mu);
  for (;;) {
    S->cv.wait(lk, [&] { return S->quit || !S->device_queue.empty(); });
    if (S->quit) return;
    Request* R = S->device_queue.front();
    S->device_queue.pop_front();
    pcg_status st = R->prep_status;
    const bool solve = st == PCG_OK;
    if (solve) {
      const pcg_status ps = pump(S);    // publishes requests whose copies have completed
      if (ps != PCG_OK) S->worker_error = ps;
      if (lanes_pending(S)) {
        S->cv.wait(lk, [&] { return S->quit || S->device_active == 0; });
        const auto defer_end = std::chrono::steady_clock::now() + kDeviceDefer;
        while (!S->quit && S->device_active == 0 && lanes_pending(S) &&
               std::chrono::steady_clock::now() < defer_end) {
          const pcg_status s = pump(S);   // publishes finished copies, (re)launches the lanes
          if (s != PCG_OK) {
            S->worker_error = s;
            break;
          }
          lk.unlock();
          std::this_thread::sleep_for(std::chrono::microseconds(200));
          lk.lock();
        }
      }
      if (S->quit) return;              // pcg_server_destroy frees the prepared context
      ++S->device_active;
      for (Lane& L : S->lane) {
        cuda::atomic_ref<unsigned, cuda::thread_scope_system> stop(L.sh->stop);
        stop.store(1u, cuda::memory_order_release);
      }
      lk.unlock();
      for (Lane& L : S->lane) {
        cuda::atomic_ref<unsigned, cuda::thread_scope_system> live(L.sh->live);
        while (live.load(cuda::memory_order_acquire) != 0) std::this_thread::sleep_for(std::chrono::microseconds(50));
        cudaStreamSynchronize(L.kstream);
      }
      R->device_res = pcg_result{};
      R->device_res.alpha_hist = R->alpha_log.data();
      R->device_res.beta_hist = R->beta_log.data();
      st = pcg_solve(R->ctx, R->b.data(), nullptr, R->method, R->method == PCG_SPCG ? R->sigma : 0.0, R->tol,
                     R->maxit, R->precision, R->x_host.data(), &R->device_res);
      // freeing device memory waits for the whole device, so the context goes while the
      // lanes are down (it may wait briefly for the other thread's queued launches)
      pcg_destroy(R->ctx);
      R->ctx = nullptr;
      lk.lock();
      --S->device_active;
    }
    R->device_status = st;
    R->device_done = true;
    release_arrays(R);
    --S->prepared;
    S->prep_cv.notify_all();
    if (S->device_active == 0) {
      const pcg_status s = pump(S);   // the lanes come back for published work
      if (s != PCG_OK) S->worker_error = s;
    }
    S->cv.notify_all();               // a thread waiting for the other's solve to end
  }
}

}  // namespace

extern "C" {

pcg_status pcg_server_create(size_t hbm_budget_bytes, int32_t max_slots, pcg_server** out) {
  if (!out) return PCG_EINVAL;
  *out = nullptr;
  if (hbm_budget_bytes < (1u << 20) || max_slots < 1 || max_slots > (1 << 20)) return PCG_EINVAL;
  pcg_server* S = new (std::nothrow) pcg_server();
  if (!S) return PCG_ENOMEM;
  auto bail = [&](pcg_status s) {
    pcg_server_destroy(S);
    return s;
  };
  if (cudaGetDevice(&S->device) != cudaSuccess) return bail(PCG_ECUDA);
  S->budget = hbm_budget_bytes & ~(size_t)255;
  S->max_slots = max_slots;
  S->cap = (unsigned)(4 * max_slots);
  void* p;
  if (cudaMalloc(&p, S->budget) != cudaSuccess) {
    cudaGetLastError();
    return bail(PCG_ENOMEM);
  }
  S->arena = (char*)p;
  S->free_blocks[0] = S->budget;
  S->stage_cap = std::min<size_t>(S->budget / 2, (size_t)128 << 20) & ~(size_t)255;
  if (cudaHostAlloc(&p, S->stage_cap, cudaHostAllocDefault) != cudaSuccess) return bail(PCG_ENOMEM);
  S->stage = (char*)p;
  if (cudaStreamCreateWithFlags(&S->cstream, cudaStreamNonBlocking) != cudaSuccess) return bail(PCG_ECUDA);
  // the GPU's resident blocks of k_server, split between the lanes
  const int small_max = server_max_clusters_t<false>(kLaneCluster[0]);
  const int large_max = server_max_clusters_wide(kLaneCluster[1]);
  if (small_max <= 0 || large_max <= 0) return bail(PCG_ECUDA);
  const int blocks = small_max * kLaneCluster[0];
  const int large = std::min(kLargeLaneClusters, std::max(1, large_max / 2));
  int host_atomics = 0;   // native atomics between the GPU and host memory (NVLink-C2C)
  if (cudaDeviceGetAttribute(&host_atomics, cudaDevAttrHostNativeAtomicSupported, S->device) != cudaSuccess) {
    cudaGetLastError();
    host_atomics = 0;
  }
  for (int l = 0; l < kLanes; ++l) {
    Lane& L = S->lane[l];
    L.csize = kLaneCluster[l];
    L.wide = l == 1;
    L.clusters = l == 1 ? large : std::max(1, (blocks - large * kLaneCluster[1]) / kLaneCluster[0]);
    L.occupied.assign(S->cap, 0);
    if (cudaHostAlloc(&p, sizeof(ServerShared), cudaHostAllocMapped) != cudaSuccess) return bail(PCG_ENOMEM);
    L.sh = (ServerShared*)p;
    memset(L.sh, 0, sizeof(ServerShared));
    L.sh->atomic_mirror = host_atomics ? 1u : 0u;
    if (cudaHostGetDevicePointer((void**)&L.d_sh, L.sh, 0) != cudaSuccess) return bail(PCG_ECUDA);
    if (cudaHostAlloc(&p, S->cap * sizeof(WorkItem), cudaHostAllocMapped) != cudaSuccess) return bail(PCG_ENOMEM);
    L.items = (WorkItem*)p;
    if (cudaHostGetDevicePointer((void**)&L.d_items, L.items, 0) != cudaSuccess) return bail(PCG_ECUDA);
    if (cudaHostAlloc(&p, S->cap * sizeof(unsigned), cudaHostAllocMapped) != cudaSuccess) return bail(PCG_ENOMEM);
    L.done = (unsigned*)p;
    memset(L.done, 0, S->cap * sizeof(unsigned));
    if (cudaHostGetDevicePointer((void**)&L.d_done, L.done, 0) != cudaSuccess) return bail(PCG_ECUDA);
    if (cudaHostAlloc(&p, S->cap * sizeof(BatchOut), cudaHostAllocMapped) != cudaSuccess) return bail(PCG_ENOMEM);
    L.results = (BatchOut*)p;
    if (cudaHostGetDevicePointer((void**)&L.d_results, L.results, 0) != cudaSuccess) return bail(PCG_ECUDA);
    if (cudaMalloc(&p, 2 * sizeof(unsigned)) != cudaSuccess) return bail(PCG_ENOMEM);
    L.d_claim = (unsigned*)p;
    L.d_left = L.d_claim + 1;
    if (cudaMemset(L.d_claim, 0, 2 * sizeof(unsigned)) != cudaSuccess) return bail(PCG_ECUDA);
    if (cudaStreamCreateWithFlags(&L.kstream, cudaStreamNonBlocking) != cudaSuccess) return bail(PCG_ECUDA);
  }
  try {
    for (std::thread& w : S->worker) w = std::thread(device_worker, S);
    S->prep = std::thread(prep_worker, S);
  } catch (...) {
    return bail(PCG_ENOMEM);
  }
  *out = S;
  return PCG_OK;
}

void pcg_server_destroy(pcg_server* S) {
  if (!S) return;
  {
    std::lock_guard<std::mutex> lock(S->mu);
    S->quit = true;
  }
  S->cv.notify_all();
  S->prep_cv.notify_all();
  for (std::thread& w : S->worker)
    if (w.joinable()) w.join();
  if (S->prep.joinable()) S->prep.join();
  for (Lane& L : S->lane) {
    if (L.sh) {
      cuda::atomic_ref<unsigned, cuda::thread_scope_system> stop(L.sh->stop);
      stop.store(1u, cuda::memory_order_release);
    }
  }
  for (Lane& L : S->lane)
    if (L.kstream) cudaStreamSynchronize(L.kstream);
  if (S->cstream) cudaStreamSynchronize(S->cstream);
  for (auto& kv : S->all) {
    if (kv.second->uploaded) cudaEventDestroy(kv.second->uploaded);
    if (kv.second->ctx) pcg_destroy(kv.second->ctx);   // prepared, never solved
    delete kv.second;
  }
  for (cudaEvent_t e : S->free_events) cudaEventDestroy(e);
  if (S->stage) cudaFreeHost(S->stage);
  if (S->arena) cudaFree(S->arena);
  for (Lane& L : S->lane) {
    if (L.d_claim) cudaFree(L.d_claim);
    if (L.sh) cudaFreeHost(L.sh);
    if (L.items) cudaFreeHost(L.items);
    if (L.done) cudaFreeHost(L.done);
    if (L.results) cudaFreeHost(L.results);
    if (L.kstream) cudaStreamDestroy(L.kstream);
  }
  if (S->cstream) cudaStreamDestroy(S->cstream);
  cudaGetLastError();
  delete S;
}

pcg_status pcg_submit(pcg_server* S, const pcg_matrix* A, const double* b, double tol, int32_t method, double sigma,
                      int32_t maxit, uint64_t* ticket) {
  return pcg_submit_ex(S, A, b, tol, method, sigma, maxit, 0, PCG_FP64, ticket);
}

pcg_status pcg_submit_ex(pcg_server* S, const pcg_matrix* A, const double* b, double tol, int32_t method,
                         double sigma, int32_t maxit, uint32_t flags, int32_t precision, uint64_t* ticket) {
  if (!S || !A || !b || !ticket) return PCG_EINVAL;
  if (method != PCG_PCG && method != PCG_SPCG) return PCG_EINVAL;
  if ((flags & ~PCG_JACOBI) || (precision != PCG_FP64 && precision != PCG_MIXED_IR)) return PCG_EINVAL;
  if (!(tol >= 0.0) || !isfinite(tol) || maxit < 0 || !isfinite(sigma)) return PCG_EINVAL;
  const int fam = family_of(*A);
  if (fam < 0) return PCG_EINVAL;
  Request* R = new (std::nothrow) Request();
  if (!R) return PCG_ENOMEM;
  R->A = *A;
  R->family = fam;
  R->tol = tol;
  R->method = method;
  R->maxit = maxit;
  R->mode = (precision == PCG_MIXED_IR ? 2 : 0) + ((flags & PCG_JACOBI) ? 1 : 0);
  const bool jac = (flags & PCG_JACOBI) != 0;
  long long n;
  double diag_sum = 0.0;
  if (fam == 4) {
    if (A->n < 1 || A->n > INT32_MAX - 64 || A->nnz < 0 || A->nnz > INT32_MAX || !A->row_ptr || !A->col || !A->val ||
        A->row_ptr[0] != 0 || A->row_ptr[A->n] != A->nnz) {
      delete R;
      return PCG_EINVAL;
    }
    n = A->n;
    R->nnz = A->nnz;
    R->row_ptr_src = A->row_ptr;
    R->col_src = A->col;
    R->val_src = A->val;
    // one pass over the rows (chunks of rows on several threads): row_ptr ranges, column
    // indices, and each row's diagonal (the sum of its diagonal entries)
    const long long nnz = A->nnz;
    std::vector<RowPass> part((size_t)host::row_chunks(n));
    host::for_chunks((long long)part.size(), [&](long long c) {
      RowPass r;
      const long long i1 = std::min(n, (c + 1) * host::kRowsPerChunk);
      for (long long i = c * host::kRowsPerChunk; i < i1 && !r.bad; ++i) {
        const long long beg = A->row_ptr[i], end = A->row_ptr[i + 1];
        if (beg < 0 || end < beg || end > nnz) {
          r.bad = true;
          break;
        }
        double dg = 0.0;
        for (long long k = beg; k < end; ++k) {
          const int32_t cj = A->col[k];
          if (cj < 0 || cj >= n) {
            r.bad = true;
            break;
          }
          if (cj == i) dg += A->val[k];
        }
        r.diag_sum += dg;
        r.diag_ok = r.diag_ok && dg > 0.0 && isfinite(dg);
      }
      part[(size_t)c] = r;
    });
    bool diag_ok = true;
    for (const RowPass& r : part) {              // in chunk order
      if (r.bad) {
        delete R;
        return PCG_EINVAL;
      }
      diag_sum += r.diag_sum;
      diag_ok = diag_ok && r.diag_ok;
    }
    if (jac && !diag_ok) {                       // Jacobi needs a positive diagonal
      delete R;
      return PCG_EINVAL;
    }
  } else {
    const long long nz = A->layout == PCG_STENCIL7_3D ? A->nz : 1;
    if (A->nx < 1 || A->ny < 1 || nz < 1 || A->nx * A->ny * nz > INT32_MAX - 64) {
      delete R;
      return PCG_EINVAL;
    }
    n = A->nx * A->ny * nz;
    if (fam == 1 || fam == 3) {
      if (!A->ax || !A->ay || (fam == 3 && !A->az)) {
        delete R;
        return PCG_EINVAL;
      }
      R->diag_src = A->diag;
      R->ax_src = A->ax;
      R->ay_src = A->ay;
      R->az_src = fam == 3 ? A->az : nullptr;
      std::vector<RowPass> part((size_t)host::row_chunks(n));
      host::for_chunks((long long)part.size(), [&](long long c) {
        RowPass r;
        const long long i1 = std::min(n, (c + 1) * host::kRowsPerChunk);
        for (long long i = c * host::kRowsPerChunk; i < i1; ++i) {
          r.diag_sum += A->diag[i];
          r.diag_ok = r.diag_ok && A->diag[i] > 0.0 && isfinite(A->diag[i]);
        }
        part[(size_t)c] = r;
      });
      bool diag_ok = true;
      for (const RowPass& r : part) {            // in chunk order
        diag_sum += r.diag_sum;
        diag_ok = diag_ok && r.diag_ok;
      }
      if (jac && !diag_ok) {
        delete R;
        return PCG_EINVAL;
      }
    } else {
      diag_sum = (double)n * (fam == 2 ? 6.0 : 4.0);
    }
  }
  R->n = n;
  // sigma < 0: the mean diagonal entry (for the unscaled Laplacians half the top of
  // the spectrum, the shift Table 1 uses for lapl200)
  // (with Jacobi, of M^{-1} A, which is 1)
  R->sigma = sigma >= 0.0 ? sigma : jac ? 1.0 : diag_sum / (double)n;
  R->b_src = b;
  R->bytes = request_bytes(*R);
  R->lane = n >= kLargeN ? 1 : 0;
  R->flags = flags;
  R->precision = precision;
  if (n >= kDeviceN) {
    R->device = true;
    own_arrays(R);                     // solved later by the device lane's thread
    std::lock_guard<std::mutex> lock(S->mu);
    if (S->worker_error != PCG_OK) {
      delete R;
      return S->worker_error;
    }
    R->ticket = S->next_ticket++;
    S->all[R->ticket] = R;
    S->prep_queue.push_back(R);
    *ticket = R->ticket;
    S->prep_cv.notify_all();
    return PCG_OK;
  }
  std::lock_guard<std::mutex> lock(S->mu);
  if (R->bytes > S->budget) {
    delete R;
    return PCG_ENOMEM;                 // can never be admitted
  }
  if (cudaSetDevice(S->device) != cudaSuccess) {
    delete R;
    return PCG_ECUDA;
  }
  R->ticket = S->next_ticket++;
  S->all[R->ticket] = R;
  S->waiting.push_back(R);
  *ticket = R->ticket;
  // admitted at once: its data went from the caller's arrays straight to staging or the
  // device; otherwise it keeps copies until memory comes free
  const pcg_status s = pump(S);
  if (!S->inflight.count(R->ticket)) own_arrays(R);
  return s;
}

pcg_status pcg_poll(pcg_server* S, uint64_t ticket, double* x_out, pcg_result* res) {
  if (!S) return PCG_EINVAL;
  std::lock_guard<std::mutex> lock(S->mu);
  auto it = S->all.find(ticket);
  if (it == S->all.end()) return PCG_EINVAL;
  Request* R = it->second;
  if (cudaSetDevice(S->device) != cudaSuccess) return PCG_ECUDA;
  pcg_status s = pump(S);
  if (s != PCG_OK) return s;
  if (R->device) {
    if (!R->device_done) return PCG_PENDING;
    const pcg_status st = R->device_status;
    if (st == PCG_OK || st == PCG_ENOTCONV || st == PCG_EBREAKDOWN) {
      if (x_out) memcpy(x_out, R->x_host.data(), (size_t)R->n * 8);
      if (res) {
        res->iters = R->device_res.iters;
        res->status = st;
        res->final_true_relres = R->device_res.final_true_relres;
        res->final_rec_relres = R->device_res.final_rec_relres;
        const int m = res->iters < kScalarLog ? res->iters : kScalarLog;
        for (int i = 0; i < m && i < (int)R->alpha_log.size(); ++i) {
          if (res->alpha_hist) res->alpha_hist[i] = R->alpha_log[i];
          if (res->beta_hist) res->beta_hist[i] = R->beta_log[i];
        }
      }
    }
    S->all.erase(it);
    delete R;
    return st;
  }
  if (R->ring < 0) return PCG_PENDING;
  const unsigned k = (unsigned)(R->ring % S->cap);
  Lane& L = S->lane[R->lane];
  cuda::atomic_ref<unsigned, cuda::thread_scope_system> d(L.done[k]);
  if (d.load(cuda::memory_order_acquire) == 0) return PCG_PENDING;
  const BatchOut o = L.results[k];
  const WorkItem& w = L.items[k];
  if (x_out && cudaMemcpyAsync(x_out, w.vec.x, (size_t)R->n * 8, cudaMemcpyDeviceToHost, S->cstream) != cudaSuccess)
    return PCG_ECUDA;
  double log[2 * kScalarLog];
  const bool want_log = res && (res->alpha_hist || res->beta_hist);
  if (want_log && cudaMemcpyAsync(log, w.sys.log, sizeof log, cudaMemcpyDeviceToHost, S->cstream) != cudaSuccess)
    return PCG_ECUDA;
  if (cudaStreamSynchronize(S->cstream) != cudaSuccess) return PCG_ECUDA;
  const pcg_status code = o.status == ST_CONVERGED ? PCG_OK : o.status == ST_BREAKDOWN ? PCG_EBREAKDOWN : PCG_ENOTCONV;
  if (res) {
    res->iters = o.iters;
    res->status = code;
    res->final_true_relres = o.bnorm > 0 ? o.true_res / o.bnorm : o.true_res;
    res->final_rec_relres = NAN;
    if (want_log) {
      const int m = o.iters < kScalarLog ? o.iters : kScalarLog;
      for (int i = 0; i < m; ++i) {
        if (res->alpha_hist) res->alpha_hist[i] = log[i];
        if (res->beta_hist) res->beta_hist[i] = log[kScalarLog + i];
      }
    }
  }
  arena_free(S, R->arena_off, R->bytes);
  L.occupied[k] = 0;
  S->inflight.erase(ticket);
  S->all.erase(it);
  delete R;
  s = pump(S);                          // memory came free: admit waiting requests
  if (s != PCG_OK) return s;
  return code;
}

pcg_status pcg_server_stats(pcg_server* S, int64_t* waiting, int64_t* inflight, size_t* free_bytes) {
  if (!S) return PCG_EINVAL;
  std::lock_guard<std::mutex> lock(S->mu);
  if (waiting) *waiting = (int64_t)(S->waiting.size() + S->prep_queue.size() + S->device_queue.size());
  if (inflight) *inflight = (int64_t)S->inflight.size();
  if (free_bytes) {
    size_t f = 0;
    for (auto& kv : S->free_blocks) f += kv.second;
    *free_bytes = f;
  }
  return PCG_OK;
}

}  // extern "C"
