// Continuous-batching query server (not in the paper, which runs one query
// at a time on one CPU thread, Section 5.1.4).
//
// Requests queue on the host.  progress() reaps batches that finished on the
// device and admits waiting requests as soon as a stream and enough device
// slots are free, so new batches start while others are still running and
// their work overlaps on the GPU.  Admission is bounded by a slot budget: the
// number of queries the search kernel can hold resident at once, which its
// shared memory per query (the query bitmap, block scores, the top-k heap of
// k entries) fixes through the occupancy calculator.  Each stream owns its
// workspace and pinned staging buffers, so concurrent batches share nothing
// but the read-only index; a query's result does not depend on what runs
// beside it.
#include <chrono>
#include <deque>
#include <thread>
#include <unordered_map>

#include "search_impl.h"


using namespace seismic;
using Clock = std::chrono::steady_clock;

namespace {

struct Request {
  uint64_t ticket;
  std::vector<uint16_t> t;
  std::vector<float> v;
  uint32_t k;
  Clock::time_point arrive;
};

struct Result {
  std::vector<uint32_t> ids;
  std::vector<float> sc;
  Clock::time_point arrive, done;
  bool finished = false;
};

template <class T> struct Pinned {
  T *p = nullptr;
  size_t n = 0;
  Pinned() = default;
  Pinned(const Pinned &) = delete;
  Pinned &operator=(const Pinned &) = delete;
  ~Pinned() { if (p) cudaFreeHost(p); }
  int ensure(size_t m) {
    if (m <= n && p) return SEISMIC_OK;
    if (p) cudaFreeHost(p);
    p = nullptr;
    n = 0;
    cudaError_t e = cudaMallocHost(&p, std::max<size_t>(m, 1) * sizeof(T));
    if (e != cudaSuccess) { p = nullptr; return cuda_fail(e, "cudaMallocHost"); }
    n = m;
    return SEISMIC_OK;
  }
};

struct Slot {
  cudaStream_t st = nullptr;
  cudaEvent_t ev = nullptr;
  Workspace ws;
  bool busy = false;
  Pinned<uint64_t> h_ip;
  Pinned<uint16_t> h_t;
  Pinned<float> h_v;
  Pinned<uint32_t> h_ids;
  Pinned<float> h_sc;
  DevBuf d_ip, d_t, d_v, d_ids, d_sc;
  std::vector<uint64_t> tickets;
  uint32_t k = 0;
};

}  // namespace

struct seismic_server {
  seismic_index *ix = nullptr;
  seismic_search_params sp{};
  seismic_server_params pp{};
  std::deque<Request> pending;
  std::unordered_map<uint64_t, Result> results;
  std::deque<Slot> slots;  // built in place: a slot owns device memory and cannot move
  std::vector<uint64_t> just_done;  // tickets the last progress() completed
  uint32_t inflight = 0, budget = 0;
  uint64_t next_ticket = 1;
  ~seismic_server() {
    for (auto &s : slots) {
      if (s.st) cudaStreamSynchronize(s.st);
      if (s.ev) cudaEventDestroy(s.ev);
      if (s.st) cudaStreamDestroy(s.st);
    }
  }
};

namespace {

int launch_batch(seismic_server *srv, Slot &s) {
  // every waiting request with the oldest request's k (a batch shares k: the
  // heap size sets the skip threshold, so mixing k would change results), in
  // arrival order, within max_batch and the slot budget
  const uint32_t k = srv->pending.front().k;
  const uint32_t room = srv->budget > srv->inflight ? srv->budget - srv->inflight : 0;
  const uint32_t cap = std::min(srv->pp.max_batch, room);
  if (cap == 0) return SEISMIC_OK;
  std::deque<Request> batch, rest;
  size_t nnz = 0;
  for (Request &r : srv->pending) {
    if (r.k == k && batch.size() < cap) {
      nnz += r.t.size();
      batch.push_back(std::move(r));
    } else {
      rest.push_back(std::move(r));
    }
  }
  srv->pending.swap(rest);
  const uint32_t n = (uint32_t)batch.size();
  int rc;
  if ((rc = s.h_ip.ensure(n + 1)) || (rc = s.h_t.ensure(nnz + 8)) || (rc = s.h_v.ensure(nnz + 4)) ||
      (rc = s.h_ids.ensure((size_t)n * k)) || (rc = s.h_sc.ensure((size_t)n * k)) ||
      (rc = s.d_ip.ensure((n + 1) * 8)) || (rc = s.d_t.ensure(nnz * 2 + 16)) || (rc = s.d_v.ensure(nnz * 4 + 16)) ||
      (rc = s.d_ids.ensure((size_t)n * k * 4)) || (rc = s.d_sc.ensure((size_t)n * k * 4))) {
    for (auto it = batch.rbegin(); it != batch.rend(); ++it) srv->pending.push_front(std::move(*it));
    return rc;
  }
  s.tickets.clear();
  size_t o = 0;
  s.h_ip.p[0] = 0;
  for (uint32_t i = 0; i < n; i++) {
    Request &r = batch[i];
    std::memcpy(s.h_t.p + o, r.t.data(), r.t.size() * 2);
    std::memcpy(s.h_v.p + o, r.v.data(), r.v.size() * 4);
    o += r.t.size();
    s.h_ip.p[i + 1] = o;
    s.tickets.push_back(r.ticket);
    Result &res = srv->results[r.ticket];
    res.arrive = r.arrive;
  }
  SZ_CUDA(cudaMemcpyAsync(s.d_ip.p, s.h_ip.p, (n + 1) * 8, cudaMemcpyHostToDevice, s.st));
  if (nnz) {
    SZ_CUDA(cudaMemcpyAsync(s.d_t.p, s.h_t.p, nnz * 2, cudaMemcpyHostToDevice, s.st));
    SZ_CUDA(cudaMemcpyAsync(s.d_v.p, s.h_v.p, nnz * 4, cudaMemcpyHostToDevice, s.st));
  }
  seismic_csr q{s.d_ip.as<uint64_t>(), s.d_t.as<uint16_t>(), s.d_v.as<float>(), n, srv->ix->dim, 1};
  seismic_search_params p = srv->sp;
  p.k = k;
  p.max_query_nnz = srv->pp.max_query_nnz;
  if ((rc = search_ws(srv->ix, &s.ws, &q, &p, s.d_ids.as<uint32_t>(), s.d_sc.as<float>(), 1, s.st, nullptr)))
    return rc;
  SZ_CUDA(cudaMemcpyAsync(s.h_ids.p, s.d_ids.p, (size_t)n * k * 4, cudaMemcpyDeviceToHost, s.st));
  SZ_CUDA(cudaMemcpyAsync(s.h_sc.p, s.d_sc.p, (size_t)n * k * 4, cudaMemcpyDeviceToHost, s.st));
  SZ_CUDA(cudaEventRecord(s.ev, s.st));
  s.k = k;
  s.busy = true;
  srv->inflight += n;
  return SEISMIC_OK;
}

int progress_impl(seismic_server *srv, uint32_t *completed) {
  uint32_t done = 0;
  srv->just_done.clear();
  for (Slot &s : srv->slots) {
    if (!s.busy) continue;
    cudaError_t e = cudaEventQuery(s.ev);
    if (e == cudaErrorNotReady) continue;
    if (e != cudaSuccess) return cuda_fail(e, "cudaEventQuery");
    const Clock::time_point now = Clock::now();
    for (size_t i = 0; i < s.tickets.size(); i++) {
      Result &r = srv->results[s.tickets[i]];
      r.ids.assign(s.h_ids.p + i * s.k, s.h_ids.p + (i + 1) * s.k);
      r.sc.assign(s.h_sc.p + i * s.k, s.h_sc.p + (i + 1) * s.k);
      r.done = now;
      r.finished = true;
      srv->just_done.push_back(s.tickets[i]);
    }
    done += (uint32_t)s.tickets.size();
    srv->inflight -= (uint32_t)s.tickets.size();
    s.busy = false;
  }
  for (Slot &s : srv->slots) {
    if (srv->pending.empty()) break;
    if (s.busy) continue;
    int rc = launch_batch(srv, s);
    if (rc) return rc;
    if (!s.busy) break;  // the slot budget is full
  }
  if (completed) *completed = done;
  return SEISMIC_OK;
}

int submit_impl(seismic_server *srv, const uint16_t *terms, const float *vals, uint32_t nnz, uint32_t k,
                Clock::time_point arrive, uint64_t *ticket) {
  if (!srv || (nnz && (!terms || !vals)) || !ticket) return fail(SEISMIC_EINVAL, "NULL argument");
  if (k == 0 || k > kMaxK) return fail(SEISMIC_EINVAL, "k must be in 1..1024");
  if (nnz > srv->pp.max_query_nnz) return fail(SEISMIC_EINVAL, "query longer than the server's max_query_nnz");
  for (uint32_t i = 0; i < nnz; i++) {
    if (terms[i] >= srv->ix->dim || (i && terms[i] <= terms[i - 1]) || !std::isfinite(vals[i]))
      return fail(SEISMIC_EINVAL, "query: terms must increase, be < dim, values finite");
  }
  Request r;
  r.ticket = srv->next_ticket++;
  r.t.assign(terms, terms + nnz);
  r.v.assign(vals, vals + nnz);
  r.k = k;
  r.arrive = arrive;
  srv->pending.push_back(std::move(r));
  *ticket = srv->next_ticket - 1;
  return SEISMIC_OK;
}

}  // namespace

extern "C" {

int seismic_server_create(seismic_index *ix, const seismic_search_params *search, const seismic_server_params *params,
                          seismic_server **out) {
  if (!ix || !search || !out) return fail(SEISMIC_EINVAL, "NULL argument");
  try {
    std::unique_ptr<seismic_server> srv(new seismic_server());
    srv->ix = ix;
    srv->sp = *search;
    if (params) srv->pp = *params;
    if (!srv->pp.max_batch) srv->pp.max_batch = 256;
    if (!srv->pp.streams) srv->pp.streams = 4;
    if (!srv->pp.max_query_nnz) srv->pp.max_query_nnz = 1024;
    if (srv->pp.streams > 64) return fail(SEISMIC_EINVAL, "at most 64 streams");
    SZ_CUDA(cudaSetDevice(ix->device));
    // slot budget: resident queries the search kernel's shared memory allows
    uint32_t budget = srv->pp.slot_budget;
    if (!budget) {
      SearchArgs a{};
      a.W = (ix->dim + 31) / 32;
      a.QN = std::max<uint32_t>(4, (srv->pp.max_query_nnz + 3) & ~3u);
      a.BMAX = std::max<uint32_t>(1, ix->max_blocks_per_list);
      a.BPOW2 = 1;
      while (a.BPOW2 < a.BMAX) a.BPOW2 <<= 1;
      a.HS = 16;
      a.CAND = 256;
      a.k = std::max<uint32_t>(search->k, 100);
      a.alpha_q = search->alpha_q;
      const uint32_t nw = search->cta_warps ? search->cta_warps : 8, g = search->group ? search->group : 1;
      a.dim = ix->dim;
      a.flat = g == 1 ? 1u : 0u;
      size_t smem = search_layout(a, nw);
      int blocks = 1;
      int rc = search_occupancy(g, nw, smem, &blocks);
      if (rc) return rc;
      int sms = 1;
      SZ_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ix->device));
      budget = (uint32_t)std::max(1, blocks) * (uint32_t)sms;
    }
    srv->budget = budget;
    for (uint32_t i = 0; i < srv->pp.streams; i++) srv->slots.emplace_back();
    for (Slot &s : srv->slots) {
      SZ_CUDA(cudaStreamCreateWithFlags(&s.st, cudaStreamNonBlocking));
      SZ_CUDA(cudaEventCreateWithFlags(&s.ev, cudaEventDisableTiming));
    }
    // warm every stream's workspace with one full batch so serving never allocates
    {
      const uint32_t n = srv->pp.max_batch;
      std::vector<uint64_t> ip(n + 1);
      std::vector<uint16_t> t(n);
      std::vector<float> v(n, 1.0f);
      for (uint32_t i = 0; i <= n; i++) ip[i] = i;
      for (Slot &s : srv->slots) {
        int rc;
        const uint32_t kk = std::max<uint32_t>(search->k, 100);
        if ((rc = s.h_ip.ensure(n + 1)) || (rc = s.h_t.ensure(4 * n + 8)) || (rc = s.h_v.ensure(4 * n + 8)) ||
            (rc = s.h_ids.ensure((size_t)n * kk)) || (rc = s.h_sc.ensure((size_t)n * kk)) ||
            (rc = s.d_ip.ensure((n + 1) * 8)) || (rc = s.d_t.ensure(8 * n + 16)) || (rc = s.d_v.ensure(16 * n + 16)) ||
            (rc = s.d_ids.ensure((size_t)n * kk * 4)) || (rc = s.d_sc.ensure((size_t)n * kk * 4)))
          return rc;
        SZ_CUDA(cudaMemcpy(s.d_ip.p, ip.data(), (n + 1) * 8, cudaMemcpyHostToDevice));
        SZ_CUDA(cudaMemcpy(s.d_t.p, t.data(), n * 2, cudaMemcpyHostToDevice));
        SZ_CUDA(cudaMemcpy(s.d_v.p, v.data(), n * 4, cudaMemcpyHostToDevice));
        seismic_csr q{s.d_ip.as<uint64_t>(), s.d_t.as<uint16_t>(), s.d_v.as<float>(), n, ix->dim, 1};
        seismic_search_params p = srv->sp;
        p.k = kk;
        p.max_query_nnz = srv->pp.max_query_nnz;
        if ((rc = search_ws(ix, &s.ws, &q, &p, s.d_ids.as<uint32_t>(), s.d_sc.as<float>(), 1, s.st, nullptr)))
          return rc;
        SZ_CUDA(cudaStreamSynchronize(s.st));
      }
    }
    *out = srv.release();
    return SEISMIC_OK;
  } catch (const std::bad_alloc &) {
    return fail(SEISMIC_ENOMEM, "host allocation failed");
  }
}

int seismic_server_submit(seismic_server *srv, const uint16_t *terms, const float *vals, uint32_t nnz, uint32_t k,
                          uint64_t *ticket) {
  try {
    return submit_impl(srv, terms, vals, nnz, k, Clock::now(), ticket);
  } catch (const std::bad_alloc &) {
    return fail(SEISMIC_ENOMEM, "host allocation failed");
  }
}

int seismic_server_progress(seismic_server *srv, uint32_t *completed) {
  if (!srv) return fail(SEISMIC_EINVAL, "NULL server");
  try {
    return progress_impl(srv, completed);
  } catch (const std::bad_alloc &) {
    return fail(SEISMIC_ENOMEM, "host allocation failed");
  }
}

int seismic_server_result(seismic_server *srv, uint64_t ticket, uint32_t *ids, float *scores, double *latency_us,
                          int32_t *done) {
  if (!srv || !done) return fail(SEISMIC_EINVAL, "NULL argument");
  auto it = srv->results.find(ticket);
  if (it == srv->results.end() || !it->second.finished) {
    *done = 0;
    if (it == srv->results.end()) {
      bool queued = false;
      for (const Request &r : srv->pending) queued |= r.ticket == ticket;
      if (!queued) return fail(SEISMIC_EINVAL, "unknown or collected ticket");
    }
    return SEISMIC_OK;
  }
  Result &r = it->second;
  if (ids) std::copy(r.ids.begin(), r.ids.end(), ids);
  if (scores) std::copy(r.sc.begin(), r.sc.end(), scores);
  if (latency_us) *latency_us = std::chrono::duration<double, std::micro>(r.done - r.arrive).count();
  *done = 1;
  srv->results.erase(it);
  return SEISMIC_OK;
}

int seismic_server_replay(seismic_server *srv, const seismic_csr *queries, const double *arrival_s,
                          const uint32_t *k_per_query, uint32_t k_stride, uint32_t *ids_out, float *scores_out,
                          double *latency_us, double *wall_s) {
  if (!srv || !queries || !arrival_s || !k_per_query || !ids_out || !scores_out || !latency_us)
    return fail(SEISMIC_EINVAL, "NULL argument");
  if (queries->on_device) return fail(SEISMIC_EINVAL, "replay takes host queries");
  const uint64_t nq = queries->n_rows;
  for (uint64_t i = 0; i < nq; i++)
    if (k_per_query[i] > k_stride) return fail(SEISMIC_EINVAL, "k_per_query above k_stride");
  try {
    std::vector<uint64_t> tick(nq);
    uint64_t next = 0, got = 0;
    const Clock::time_point t0 = Clock::now();
    while (got < nq) {
      const double now = std::chrono::duration<double>(Clock::now() - t0).count();
      while (next < nq && arrival_s[next] <= now) {
        const uint64_t a = queries->indptr[next], b = queries->indptr[next + 1];
        const Clock::time_point when =
            t0 + std::chrono::duration_cast<Clock::duration>(std::chrono::duration<double>(arrival_s[next]));
        int rc = submit_impl(srv, queries->terms + a, queries->vals + a, (uint32_t)(b - a), k_per_query[next], when,
                             &tick[next]);
        if (rc) return rc;
        next++;
      }
      uint32_t done = 0;
      int rc = progress_impl(srv, &done);
      if (rc) return rc;
      if (done) {
        for (uint64_t t : srv->just_done) {
          const uint64_t i = t - tick[0];  // tickets are issued in submission order
          if (i >= next || tick[i] != t) continue;
          auto it = srv->results.find(t);
          Result &r = it->second;
          const uint32_t k = k_per_query[i];
          for (uint32_t j = 0; j < k_stride; j++) {
            ids_out[i * k_stride + j] = j < k ? r.ids[j] : SEISMIC_NONE_ID;
            scores_out[i * k_stride + j] = j < k ? r.sc[j] : -INFINITY;
          }
          latency_us[i] = std::chrono::duration<double, std::micro>(r.done - r.arrive).count();
          srv->results.erase(it);
          got++;
        }
      } else if (next < nq && srv->pending.empty() && srv->inflight == 0) {
        std::this_thread::yield();
      }
    }
    if (wall_s) *wall_s = std::chrono::duration<double>(Clock::now() - t0).count();
    return SEISMIC_OK;
  } catch (const std::bad_alloc &) {
    return fail(SEISMIC_ENOMEM, "host allocation failed");
  }
}

void seismic_server_destroy(seismic_server *srv) { delete srv; }

}  // extern "C"
