// Batch runtime: continuous batching of solve requests over resident domains,
// admitted against a caller-owned device memory pool (the serving form of
// Alg. "fft_dd_solver").
//
// A request is a domain descriptor (its nrhs = the request's right-hand
// sides), a device pointer to those right-hand sides and one for the
// solutions.  Requests with the same descriptor (apart from nrhs) form one
// queue and are served by resident domains of that descriptor with `slots`
// right-hand sides each: an idle domain takes the oldest queued requests whose
// right-hand sides fit its slots and solves them in one batch (unused slots
// carry zero and converge at once).  While every domain of a busy descriptor is
// solving and its queue is not empty, another domain of it is created if the
// pool has room (up to max_per_key).  Each domain has its own CUDA stream, so
// batches overlap on the device.
// fpg_batch_step never waits for the device: it advances every domain whose
// last enqueued stage has finished (CUDA event query) and starts idle domains.
// Domain workspaces and solution buffers are carved first-fit from the pool;
// when a new key does not fit, idle domains are evicted least recently used
// first, and a request that still does not fit is refused (FPG_EBUDGET).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <deque>
#include <new>
#include <unordered_map>
#include <vector>

#include "fpg_internal.cuh"
#include "fpg_pool.h"

namespace fpg {

fpg_status batch_start(fpg_domain* D, double* p);
bool batch_ready(fpg_domain* D);
fpg_status batch_advance(fpg_domain* D, bool* finished);
fpg_status batch_info(fpg_domain* D, fpg_solve_info* info);
fpg_status batch_zero_rhs(fpg_domain* D, int first);

namespace {

struct Request {
  int64_t ticket;
  const double* f;
  double* p;
  int nrhs;
};

enum class DomState { Idle, Running, Copying };

struct KeyQueue {
  fpg_domain_desc key;  // nrhs = slots
  std::deque<Request> pending;
  int residents = 0;
};

struct Resident {
  fpg_domain_desc key;  // nrhs = slots
  KeyQueue* kq = nullptr;
  fpg_domain* d = nullptr;
  cudaStream_t st = nullptr;
  cudaEvent_t copied = nullptr;
  size_t off = 0, bytes = 0;  // pool range (workspace, then the solution buffer)
  double* pbuf = nullptr;
  long long ntot = 0;
  DomState state = DomState::Idle;
  std::vector<Request> running;
  std::vector<fpg_solve_info> infos;  // one per slot, from the last finished batch
  uint64_t last_used = 0;
};

struct TicketState {
  bool done = false;
  std::vector<fpg_solve_info> info;
};

bool same_key(const fpg_domain_desc& a, const fpg_domain_desc& b) {
  return a.geometry == b.geometry && a.n == b.n && a.kappa == b.kappa && a.restart == b.restart &&
         a.rtol == b.rtol && a.max_iters == b.max_iters && a.precond_precision == b.precond_precision &&
         a.schur_mode == b.schur_mode && a.boundary == b.boundary && a.chain == b.chain && a.lattice == b.lattice;
}

}  // namespace
}  // namespace fpg

struct fpg_batch {
  int slots = 0, max_domains = 0, max_per_key = 0, max_busy = 0;
  std::vector<fpg::KeyQueue*> keys;
  char* pool = nullptr;
  size_t pool_bytes = 0;
  fpg::PoolFreeList free_list;  // (offset, bytes) ranges, sorted, coalesced
  std::vector<fpg::Resident*> doms;
  std::unordered_map<int64_t, fpg::TicketState> tickets;
  int64_t next_ticket = 1;
  uint64_t clock = 0;
  long long created = 0, evicted = 0;
};

namespace fpg {
namespace {

void drop_resident(fpg_batch* b, size_t idx) {
  Resident* R = b->doms[idx];
  R->kq->residents--;
  cudaStreamSynchronize(R->st);
  fpg_destroy_domain(R->d);
  cudaEventDestroy(R->copied);
  cudaStreamDestroy(R->st);
  b->free_list.give(R->off, R->bytes);
  delete R;
  b->doms.erase(b->doms.begin() + idx);
}

// Evict the least recently used idle domain with no pending work; false if none.
bool evict_one(fpg_batch* b) {
  size_t best = b->doms.size();
  for (size_t i = 0; i < b->doms.size(); ++i) {
    const Resident* R = b->doms[i];
    if (R->state != DomState::Idle || !R->kq->pending.empty()) continue;
    if (best == b->doms.size() || R->last_used < b->doms[best]->last_used) best = i;
  }
  if (best == b->doms.size()) return false;
  drop_resident(b, best);
  b->evicted++;
  return true;
}

fpg_status make_resident(fpg_batch* b, KeyQueue* kq, bool may_evict, Resident** out) {
  const fpg_domain_desc& key = kq->key;
  size_t ws = 0;
  FPG_TRY(fpg_workspace_bytes(&key, &ws));
  int64_t ntot = 0;
  FPG_TRY(fpg_unknowns(&key, &ntot));
  const size_t pbytes = sizeof(double) * (size_t)key.nrhs * (size_t)ntot;
  const size_t need = align256(ws) + align256(pbytes);
  if (need > b->pool_bytes) return FPG_EBUDGET;
  size_t off = 0;
  for (;;) {
    if ((int)b->doms.size() < b->max_domains && b->free_list.take(need, &off)) break;
    if (!may_evict || !evict_one(b)) return FPG_EBUDGET;
  }
  Resident* R = new (std::nothrow) Resident();
  if (!R) {
    b->free_list.give(off, need);
    return FPG_ENOMEM;
  }
  R->key = key;
  R->kq = kq;
  R->off = off;
  R->bytes = need;
  R->ntot = ntot;
  R->pbuf = reinterpret_cast<double*>(b->pool + off + align256(ws));
  R->infos.resize(key.nrhs);
  cudaError_t e = cudaStreamCreateWithFlags(&R->st, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&R->copied, cudaEventDisableTiming);
  fpg_status s = e == cudaSuccess ? fpg_create_domain(&key, b->pool + off, ws, R->st, &R->d) : FPG_ECUDA;
  if (s != FPG_OK) {
    if (e != cudaSuccess) record_cuda_error(e, "fpg_batch_admit");
    if (R->copied) cudaEventDestroy(R->copied);
    if (R->st) cudaStreamDestroy(R->st);
    b->free_list.give(off, need);
    delete R;
    return s;
  }
  b->doms.push_back(R);
  kq->residents++;
  b->created++;
  *out = R;
  return FPG_OK;
}

// An idle domain takes the oldest queued requests of its key that fit its slots and starts.
fpg_status start_batch(fpg_batch* b, Resident* R) {
  int used = 0;
  std::deque<Request>& q = R->kq->pending;
  while (!q.empty() && used + q.front().nrhs <= R->key.nrhs) {
    R->running.push_back(q.front());
    used += q.front().nrhs;
    q.pop_front();
  }
  if (R->running.empty()) return FPG_OK;
  int slot = 0;
  for (const Request& q : R->running) {
    for (int i = 0; i < q.nrhs; ++i, ++slot)
      FPG_TRY(fpg_set_rhs(R->d, q.f + (size_t)i * R->ntot, slot));
  }
  FPG_TRY(batch_zero_rhs(R->d, slot));
  FPG_TRY(batch_start(R->d, R->pbuf));
  R->state = DomState::Running;
  R->last_used = ++b->clock;
  return FPG_OK;
}

}  // namespace
}  // namespace fpg

using namespace fpg;

extern "C" {

fpg_status fpg_batch_create(const fpg_batch_desc* desc, void* pool, size_t pool_bytes, fpg_batch** out) {
  if (!desc || !pool || !out || desc->slots < 1 || desc->slots > 64 || desc->max_domains < 1 ||
      desc->max_domains > 256 || desc->max_per_key < 0 || desc->max_per_key > 16 || desc->max_busy < 0)
    return FPG_EINVAL;
  fpg_batch* b = new (std::nothrow) fpg_batch();
  if (!b) return FPG_ENOMEM;
  b->slots = desc->slots;
  b->max_domains = desc->max_domains;
  b->max_per_key = desc->max_per_key > 0 ? desc->max_per_key : 4;
  b->max_busy = desc->max_busy > 0 ? desc->max_busy : 1 << 30;
  // the pool starts at a 256-byte boundary
  const uintptr_t base = reinterpret_cast<uintptr_t>(pool);
  const size_t skip = (256 - base % 256) % 256;
  if (pool_bytes <= skip) {
    delete b;
    return FPG_ENOMEM;
  }
  b->pool = static_cast<char*>(pool) + skip;
  b->pool_bytes = (pool_bytes - skip) & ~(size_t)255;
  b->free_list.reset(b->pool_bytes);
  *out = b;
  return FPG_OK;
}

fpg_status fpg_batch_admit(fpg_batch* b, const fpg_domain_desc* req, const double* f_dev, double* p_dev,
                           int64_t* ticket) {
  if (!b || !req || !f_dev || !p_dev || !ticket || req->nrhs < 1 || req->nrhs > b->slots) return FPG_EINVAL;
  fpg_domain_desc key = *req;
  key.nrhs = b->slots;
  size_t ws = 0;
  FPG_TRY(fpg_workspace_bytes(&key, &ws));  // descriptor errors before anything is queued
  KeyQueue* kq = nullptr;
  for (KeyQueue* x : b->keys)
    if (same_key(x->key, key)) {
      kq = x;
      break;
    }
  if (!kq) {
    kq = new (std::nothrow) KeyQueue();
    if (!kq) return FPG_ENOMEM;
    kq->key = key;
    b->keys.push_back(kq);
  }
  if (kq->residents == 0) {  // the key needs one domain to make progress
    Resident* R = nullptr;
    FPG_TRY(make_resident(b, kq, true, &R));
  }
  const int64_t t = b->next_ticket++;
  kq->pending.push_back(Request{t, f_dev, p_dev, req->nrhs});
  b->tickets[t] = TicketState{};
  *ticket = t;
  return FPG_OK;
}

fpg_status fpg_batch_step(fpg_batch* b, int64_t* finished_tickets, int32_t cap, int32_t* completed) {
  if (!b || cap < 0 || (cap > 0 && !finished_tickets)) return FPG_EINVAL;
  int done = 0;
  for (Resident* R : b->doms) {
    if (R->state == DomState::Running && batch_ready(R->d)) {
      bool finished = false;
      FPG_TRY(batch_advance(R->d, &finished));
      if (finished) {
        const fpg_status s = batch_info(R->d, R->infos.data());
        if (s != FPG_OK && s != FPG_ENOCONV) return s;
        int slot = 0;
        for (const Request& q : R->running) {
          FPG_CUDA_TRY(cudaMemcpyAsync(q.p, R->pbuf + (size_t)slot * R->ntot,
                                       sizeof(double) * (size_t)q.nrhs * R->ntot, cudaMemcpyDeviceToDevice, R->st));
          slot += q.nrhs;
        }
        FPG_CUDA_TRY(cudaEventRecord(R->copied, R->st));
        R->state = DomState::Copying;
      }
    }
    if (R->state == DomState::Copying && cudaEventQuery(R->copied) == cudaSuccess) {
      int slot = 0;
      for (const Request& q : R->running) {
        TicketState& ts = b->tickets[q.ticket];
        ts.info.assign(R->infos.begin() + slot, R->infos.begin() + slot + q.nrhs);
        ts.done = true;
        slot += q.nrhs;
        if (done < cap) finished_tickets[done] = q.ticket;
        ++done;
      }
      R->running.clear();
      R->state = DomState::Idle;
    }
  }
  // start batches, oldest queued request first, while fewer than max_busy
  // domains are solving; a key whose domains are all busy gets one more domain
  // from free pool space (no eviction: that would trade one key's domain for
  // another's creation)
  int busy = 0;
  for (const Resident* R : b->doms) busy += R->state != DomState::Idle;
  std::vector<KeyQueue*> order;
  for (KeyQueue* kq : b->keys)
    if (!kq->pending.empty()) order.push_back(kq);
  std::sort(order.begin(), order.end(),
            [](const KeyQueue* x, const KeyQueue* y) { return x->pending.front().ticket < y->pending.front().ticket; });
  for (KeyQueue* kq : order) {
    while (busy < b->max_busy && !kq->pending.empty()) {
      Resident* R = nullptr;
      for (Resident* x : b->doms)
        if (x->kq == kq && x->state == DomState::Idle) {
          R = x;
          break;
        }
      if (!R && (kq->residents >= b->max_per_key || make_resident(b, kq, false, &R) != FPG_OK)) break;
      FPG_TRY(start_batch(b, R));
      ++busy;
    }
  }
  if (completed) *completed = done;
  return FPG_OK;
}

fpg_status fpg_batch_poll(fpg_batch* b, int64_t ticket, int32_t* done, fpg_solve_info* info) {
  if (!b || !done) return FPG_EINVAL;
  auto it = b->tickets.find(ticket);
  if (it == b->tickets.end()) return FPG_EINVAL;
  *done = it->second.done ? 1 : 0;
  if (it->second.done) {
    if (info) std::memcpy(info, it->second.info.data(), sizeof(fpg_solve_info) * it->second.info.size());
    b->tickets.erase(it);
  }
  return FPG_OK;
}

fpg_status fpg_batch_stats(fpg_batch* b, fpg_batch_stats_t* out) {
  if (!b || !out) return FPG_EINVAL;
  std::memset(out, 0, sizeof(*out));
  out->resident = (int32_t)b->doms.size();
  for (const Resident* R : b->doms) {
    out->pool_used += (int64_t)R->bytes;
    if (R->state != DomState::Idle) out->busy++;
  }
  for (const KeyQueue* kq : b->keys) out->queued += (int32_t)kq->pending.size();
  for (const auto& kv : b->tickets) out->open_tickets += kv.second.done ? 0 : 1;
  out->created = b->created;
  out->evicted = b->evicted;
  return FPG_OK;
}

void fpg_batch_destroy(fpg_batch* b) {
  if (!b) return;
  while (!b->doms.empty()) drop_resident(b, b->doms.size() - 1);
  for (KeyQueue* kq : b->keys) delete kq;
  delete b;
}

}  // extern "C"
