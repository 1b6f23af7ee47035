// sched.cpp - region-driven asynchronous scheduling of device work.
//
// The runtime tracks the memory range every submitted task reads and writes
// and lets tasks whose ranges do not conflict run at the same time on a pool
// of streams; a task waits (cudaStreamWaitEvent) only for earlier tasks it
// conflicts with: read after write, write after read or write after write on
// overlapping bytes (§3.2.1 tracks the range each kernel touches, §4 runs
// kernels asynchronously, §6.1 uses 16 queues).  A task's ranges come from
// region analysis of its loop nest (jacc_region_analyze: the exact flattened
// offset extremes of every array it touches), from a stencil sweep's two
// fields, or from a copy's source and destination.
//
// Dependencies come from an interval map over the bytes tasks have touched:
// disjoint segments, each holding its last writer and the tasks that read it
// since.  A reading range depends on the last writers of the segments it
// overlaps; a writing range also on their readers.  Those tasks are the only
// ones a new task must wait for: every earlier conflicting task is ordered
// before one of them already.  A query costs O(log n + segments overlapped).
//
// In dry-run mode no CUDA call is made: the scheduler only records each
// task's dependencies and stream, so the dependency logic can be checked on
// a host without a GPU.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstddef>
#include <cstring>
#include <iterator>
#include <map>
#include <mutex>
#include <vector>

#include "jacc_internal.h"

namespace jacc {
namespace {

struct Range {
  uint64_t lo, hi;  // bytes [lo, hi)
  bool write;
};

struct Task {
  std::vector<Range> ranges;
  std::vector<int32_t> deps;  // earlier tasks this one waits for
  int32_t stream = -1;
  cudaEvent_t done = nullptr;  // recorded after the task's work (live mode)
  bool open = false;           // a nest task between begin and end
  bool retired = false;        // completed on the device: no later task needs to wait for it
};

// A segment [key, hi) of touched bytes.
struct Seg {
  uint64_t hi;
  int32_t writer;                // last task that wrote it (-1: none)
  std::vector<int32_t> readers;  // tasks that read it since that write
};
typedef std::map<uint64_t, Seg> SegMap;

// The first segment that overlaps [lo, ...).
SegMap::iterator first_overlap(SegMap& m, uint64_t lo) {
  auto it = m.upper_bound(lo);
  if (it != m.begin()) {
    auto p = std::prev(it);
    if (p->second.hi > lo) return p;
  }
  return it;
}

// Splits the segment holding x, if any, so that a segment starts at x.
void cut(SegMap& m, uint64_t x) {
  auto it = m.upper_bound(x);
  if (it == m.begin()) return;
  --it;
  if (it->first < x && x < it->second.hi) {
    Seg right = it->second;
    it->second.hi = x;
    m.emplace(x, std::move(right));
  }
}

// Records that task `id` reads (write = false) or writes [lo, hi).
void record(SegMap& m, uint64_t lo, uint64_t hi, bool write, int32_t id) {
  cut(m, lo);
  cut(m, hi);
  auto apply = [&](Seg& g) {
    if (write) {
      g.writer = id;
      g.readers.clear();
    } else if (std::find(g.readers.begin(), g.readers.end(), id) == g.readers.end()) {
      g.readers.push_back(id);
    }
  };
  uint64_t pos = lo;
  auto it = m.lower_bound(lo);
  while (pos < hi) {
    if (it == m.end() || it->first > pos) {  // untouched bytes [pos, end)
      const uint64_t end = (it == m.end() || it->first > hi) ? hi : it->first;
      Seg g{end, -1, {}};
      apply(g);
      it = std::next(m.emplace_hint(it, pos, std::move(g)));
      pos = end;
      continue;
    }
    apply(it->second);
    pos = it->second.hi;
    ++it;
  }
  if (write) {  // the written segments now agree: merge them
    auto a = m.find(lo);
    while (a != m.end() && a->first < hi) {
      auto b = std::next(a);
      if (b != m.end() && b->first == a->second.hi && b->first < hi && b->second.writer == id &&
          b->second.readers.empty()) {
        a->second.hi = b->second.hi;
        m.erase(b);
      } else {
        a = b;
      }
    }
  }
}

}  // namespace

struct Sched {
  bool dry = false;
  std::vector<cudaStream_t> streams;
  std::vector<int32_t> last_task;  // per stream: the last task placed on it (-1: none)
  std::vector<Task> tasks;
  SegMap segs;            // the dependency index
  std::vector<int32_t> pending;  // live mode: tasks to retire once completed (submission order, plus
                                 // former stream anchors and closed nests queued again)
  size_t pending_head = 0;       // first entry of `pending` still to check
  int64_t live_events = 0;       // tasks whose completion event still exists
  int32_t next_free = 0;  // round-robin cursor for tasks without dependencies
  std::mutex mu;
};

// Live mode: retires the oldest tasks that have completed on the device
// (their events are destroyed; a later task that names them waits for
// nothing).  Stops at the first task still running, so the cost stays
// proportional to the tasks passed.  A stream's last task (the anchor of its
// chain, whose event jacc_sched_join waits on) and an open nest task cannot
// be retired yet: they leave the queue here and are queued again when they
// stop being one (place() when the stream gets a new last task,
// jacc_sched_nest_end when the nest closes), so every task is retired once
// it has completed and is neither.
static void retire_completed(Sched& s) {
  while (s.pending_head < s.pending.size()) {
    const int32_t j = s.pending[s.pending_head];
    Task& o = s.tasks[j];
    if (!o.retired && !o.open && o.done && s.last_task[o.stream] != j) {
      if (cudaEventQuery(o.done) != cudaSuccess) break;
      cudaEventDestroy(o.done);
      o.done = nullptr;
      o.retired = true;
      --s.live_events;
    }
    ++s.pending_head;
  }
  if (s.pending_head > 4096 && s.pending_head * 2 > s.pending.size()) {
    s.pending.erase(s.pending.begin(), s.pending.begin() + static_cast<std::ptrdiff_t>(s.pending_head));
    s.pending_head = 0;
  }
}

static jacc_status place(Sched& s, std::vector<Range> ranges, int32_t* id_out, cudaStream_t* stream_out) {
  if (!s.dry) retire_completed(s);
  Task t;
  t.ranges = std::move(ranges);
  const int32_t id = static_cast<int32_t>(s.tasks.size());
  std::vector<int32_t> cand;
  for (const Range& r : t.ranges) {
    if (r.lo >= r.hi) continue;
    for (auto it = first_overlap(s.segs, r.lo); it != s.segs.end() && it->first < r.hi; ++it) {
      if (it->second.writer >= 0) cand.push_back(it->second.writer);
      if (r.write) cand.insert(cand.end(), it->second.readers.begin(), it->second.readers.end());
    }
  }
  std::sort(cand.begin(), cand.end());
  cand.erase(std::unique(cand.begin(), cand.end()), cand.end());
  for (int32_t j : cand) {
    Task& o = s.tasks[j];
    if (o.retired) continue;
    if (!s.dry && !o.open && o.done && s.last_task[o.stream] != j && cudaEventQuery(o.done) == cudaSuccess) {
      // finished on the device: drop it (its stream's last task is kept as
      // the chain anchor)
      cudaEventDestroy(o.done);
      o.done = nullptr;
      o.retired = true;
      --s.live_events;
      continue;
    }
    t.deps.push_back(j);
  }
  // stream: continue the chain of the latest dependency if it ends its
  // stream (no wait needed for it); otherwise the next stream round-robin
  int32_t st = -1;
  if (!t.deps.empty()) {
    const int32_t d = t.deps.back();
    const int32_t ds = s.tasks[d].stream;
    if (ds >= 0 && s.last_task[ds] == d) st = ds;
  }
  if (st < 0) {
    st = s.next_free;
    s.next_free = (s.next_free + 1) % static_cast<int32_t>(s.last_task.size());
  }
  t.stream = st;
  if (!s.dry) {
    for (int32_t d : t.deps) {
      if (s.tasks[d].stream == st) continue;  // stream order already covers it
      if (s.tasks[d].open) return fail(JACC_ERR_INVALID_ARG, "a dependency is a nest task that was not ended");
      jacc_status e = cuda_check(cudaStreamWaitEvent(s.streams[st], s.tasks[d].done, 0), "cudaStreamWaitEvent");
      if (e) return e;
    }
    jacc_status e = cuda_check(cudaEventCreateWithFlags(&t.done, cudaEventDisableTiming), "cudaEventCreate");
    if (e) return e;
    ++s.live_events;
  }
  // the task is placed: enter its ranges into the index (reads first, so a
  // range both read and written ends as written)
  for (const Range& r : t.ranges)
    if (!r.write && r.lo < r.hi) record(s.segs, r.lo, r.hi, false, id);
  for (const Range& r : t.ranges)
    if (r.write && r.lo < r.hi) record(s.segs, r.lo, r.hi, true, id);
  // the stream's previous last task stops being its anchor: queue it again
  // (it completes before the new task, which follows it on the stream)
  const int32_t old_anchor = s.last_task[st];
  if (!s.dry && old_anchor >= 0 && !s.tasks[old_anchor].retired) s.pending.push_back(old_anchor);
  s.last_task[st] = id;
  s.tasks.push_back(std::move(t));
  if (!s.dry) s.pending.push_back(id);
  *id_out = id;
  if (stream_out) *stream_out = s.dry ? nullptr : s.streams[st];
  return ok();
}

static jacc_status finish(Sched& s, int32_t id) {
  if (s.dry) return ok();
  Task& t = s.tasks[id];
  return cuda_check(cudaEventRecord(t.done, s.streams[t.stream]), "cudaEventRecord");
}

}  // namespace jacc

using namespace jacc;

extern "C" jacc_status jacc_sched_create(int32_t nstreams, uint32_t flags, uintptr_t origin, jacc_sched* out) {
  if (!out || nstreams < 1 || nstreams > 64) return fail(JACC_ERR_INVALID_ARG, "nstreams must be in [1, 64]");
  if (flags & ~JACC_SCHED_DRY_RUN) return fail(JACC_ERR_INVALID_ARG, "unknown scheduler flags");
  Sched* s = new Sched();
  s->dry = (flags & JACC_SCHED_DRY_RUN) != 0;
  s->last_task.assign(nstreams, -1);
  if (!s->dry) {
    cudaEvent_t start = nullptr;
    jacc_status st = cuda_check(cudaEventCreateWithFlags(&start, cudaEventDisableTiming), "cudaEventCreate");
    if (!st) st = cuda_check(cudaEventRecord(start, reinterpret_cast<cudaStream_t>(origin)), "cudaEventRecord");
    for (int32_t i = 0; !st && i < nstreams; ++i) {
      cudaStream_t c = nullptr;
      st = cuda_check(cudaStreamCreateWithFlags(&c, cudaStreamNonBlocking), "cudaStreamCreate");
      if (!st) {
        s->streams.push_back(c);
        // the pool starts after the work already queued on the origin stream
        st = cuda_check(cudaStreamWaitEvent(c, start, 0), "cudaStreamWaitEvent");
      }
    }
    if (start) cudaEventDestroy(start);
    if (st) {
      for (cudaStream_t c : s->streams) cudaStreamDestroy(c);
      delete s;
      return st;
    }
  }
  *out = reinterpret_cast<jacc_sched>(s);
  return ok();
}

extern "C" jacc_status jacc_sched_sweep(jacc_sched h, jacc_kernel k, void* u0, void* u1, int32_t nsweeps,
                                        double* resid_dev, int32_t* task_id) {
  if (!h || !k || !task_id) return fail(JACC_ERR_INVALID_ARG, "NULL scheduler, kernel or task_id");
  Sched& s = *reinterpret_cast<Sched*>(h);
  const Kernel& kk = *reinterpret_cast<Kernel*>(k);
  if (nsweeps < 1) return fail(JACC_ERR_INVALID_ARG, "nsweeps must be >= 1");
  jacc_status st = check_buffers(kk, u0, u1);
  if (st) return st;
  // the sweep's regions: every point of the input is read (interior points
  // by the stencil, boundary points by the copy) and every point of the
  // output written; from two sweeps on, both fields are read and written
  const uint64_t bytes = static_cast<uint64_t>(kk.desc.nx * kk.desc.ny * kk.desc.nz) * kk.elem;
  const uint64_t a = reinterpret_cast<uint64_t>(u0), b = reinterpret_cast<uint64_t>(u1);
  std::vector<Range> r = {{a, a + bytes, false}, {b, b + bytes, true}};
  if (nsweeps >= 2) {
    r.push_back({a, a + bytes, true});
    r.push_back({b, b + bytes, false});
  }
  if (resid_dev) {
    const uint64_t q = reinterpret_cast<uint64_t>(resid_dev);
    r.push_back({q, q + sizeof(double) * static_cast<uint64_t>(nsweeps), true});
  }
  std::lock_guard<std::mutex> lock(s.mu);
  cudaStream_t cs = nullptr;
  int32_t id = -1;
  st = place(s, std::move(r), &id, &cs);
  if (st) return st;
  if (!s.dry) {
    int32_t fb = 0;
    st = jacc_sweep(k, u0, u1, nsweeps, resid_dev, JACC_SWEEP_GRAPH, reinterpret_cast<uintptr_t>(cs), &fb);
    if (st) return st;
  }
  *task_id = id;
  return finish(s, id);
}

extern "C" jacc_status jacc_sched_copy(jacc_sched h, void* dst, const void* src, uint64_t bytes, int32_t* task_id) {
  if (!h || !dst || !src || !task_id) return fail(JACC_ERR_INVALID_ARG, "NULL argument");
  Sched& s = *reinterpret_cast<Sched*>(h);
  const uint64_t d = reinterpret_cast<uint64_t>(dst), c = reinterpret_cast<uint64_t>(src);
  if (d < c + bytes && c < d + bytes) return fail(JACC_ERR_INVALID_ARG, "copy source and destination overlap");
  std::lock_guard<std::mutex> lock(s.mu);
  cudaStream_t cs = nullptr;
  int32_t id = -1;
  jacc_status st = place(s, {{c, c + bytes, false}, {d, d + bytes, true}}, &id, &cs);
  if (st) return st;
  if (!s.dry) {
    st = cuda_check(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, cs), "cudaMemcpyAsync");
    if (st) return st;
  }
  *task_id = id;
  return finish(s, id);
}

// A nest task from the regions its loop nest touches (analysed by the caller).
static jacc_status nest_task(jacc_sched h, const std::vector<jacc_region>& reg, int32_t narrays, const uint64_t* base,
                             const int32_t* elem_bytes, int32_t* task_id, uintptr_t* stream_out) {
  Sched& s = *reinterpret_cast<Sched*>(h);
  jacc_status st = ok();
  std::vector<Range> r;
  for (int32_t a = 0; a < narrays; ++a) {
    if (elem_bytes[a] < 1) return fail(JACC_ERR_INVALID_ARG, "elem_bytes must be >= 1");
    const uint64_t e = static_cast<uint64_t>(elem_bytes[a]);
    if (reg[a].has_read)
      r.push_back({base[a] + static_cast<uint64_t>(reg[a].rlin_lo) * e, base[a] + static_cast<uint64_t>(reg[a].rlin_hi + 1) * e,
                   false});
    if (reg[a].has_write)
      r.push_back({base[a] + static_cast<uint64_t>(reg[a].wlin_lo) * e, base[a] + static_cast<uint64_t>(reg[a].wlin_hi + 1) * e,
                   true});
  }
  std::lock_guard<std::mutex> lock(s.mu);
  cudaStream_t cs = nullptr;
  int32_t id = -1;
  st = place(s, std::move(r), &id, &cs);
  if (st) return st;
  s.tasks[id].open = true;
  *task_id = id;
  *stream_out = reinterpret_cast<uintptr_t>(cs);
  return ok();
}

extern "C" jacc_status jacc_sched_nest_begin(jacc_sched h, int32_t nloops, const jacc_loop* loops, int32_t nrefs,
                                             const jacc_ref* refs, int32_t narrays, const jacc_array* arrays,
                                             const uint64_t* base, const int32_t* elem_bytes, int32_t* task_id,
                                             uintptr_t* stream_out) {
  if (!h || !task_id || !stream_out || (narrays > 0 && (!base || !elem_bytes)))
    return fail(JACC_ERR_INVALID_ARG, "NULL argument");
  if (narrays < 0 || narrays > 64) return fail(JACC_ERR_INVALID_ARG, "narrays must be in [0, 64]");
  std::vector<jacc_region> reg(static_cast<size_t>(narrays));
  jacc_status st = jacc_region_analyze(nloops, loops, nrefs, refs, narrays, arrays, reg.data());
  if (st) return st;
  return nest_task(h, reg, narrays, base, elem_bytes, task_id, stream_out);
}

extern "C" jacc_status jacc_sched_nest_begin_affine(jacc_sched h, int32_t nloops, const jacc_loop_affine* loops,
                                                    int32_t nrefs, const jacc_ref* refs, int32_t narrays,
                                                    const jacc_array* arrays, const uint64_t* base,
                                                    const int32_t* elem_bytes, int32_t* task_id,
                                                    uintptr_t* stream_out) {
  if (!h || !task_id || !stream_out || (narrays > 0 && (!base || !elem_bytes)))
    return fail(JACC_ERR_INVALID_ARG, "NULL argument");
  if (narrays < 0 || narrays > 64) return fail(JACC_ERR_INVALID_ARG, "narrays must be in [0, 64]");
  std::vector<jacc_region> reg(static_cast<size_t>(narrays));
  jacc_status st = jacc_region_analyze_affine(nloops, loops, nrefs, refs, narrays, arrays, reg.data());
  if (st) return st;
  return nest_task(h, reg, narrays, base, elem_bytes, task_id, stream_out);
}

extern "C" jacc_status jacc_sched_nest_end(jacc_sched h, int32_t task_id) {
  if (!h) return fail(JACC_ERR_INVALID_ARG, "NULL scheduler");
  Sched& s = *reinterpret_cast<Sched*>(h);
  std::lock_guard<std::mutex> lock(s.mu);
  if (task_id < 0 || task_id >= static_cast<int32_t>(s.tasks.size()) || !s.tasks[task_id].open)
    return fail(JACC_ERR_INVALID_ARG, "not an open nest task");
  s.tasks[task_id].open = false;
  if (!s.dry) s.pending.push_back(task_id);  // retirable once completed
  return finish(s, task_id);
}

extern "C" jacc_status jacc_sched_task_info(jacc_sched h, int32_t task_id, int32_t* deps, int32_t max_deps,
                                            int32_t* ndeps, int32_t* stream_index) {
  if (!h || !ndeps || !stream_index || (max_deps > 0 && !deps)) return fail(JACC_ERR_INVALID_ARG, "NULL argument");
  Sched& s = *reinterpret_cast<Sched*>(h);
  std::lock_guard<std::mutex> lock(s.mu);
  if (task_id < 0 || task_id >= static_cast<int32_t>(s.tasks.size())) return fail(JACC_ERR_INVALID_ARG, "bad task_id");
  const Task& t = s.tasks[task_id];
  *ndeps = static_cast<int32_t>(t.deps.size());
  *stream_index = t.stream;
  for (int32_t i = 0; i < max_deps && i < *ndeps; ++i) deps[i] = t.deps[i];
  return ok();
}

extern "C" jacc_status jacc_sched_live_events(jacc_sched h, int64_t* live_events, int64_t* ntasks) {
  if (!h || !live_events) return fail(JACC_ERR_INVALID_ARG, "NULL argument");
  Sched& s = *reinterpret_cast<Sched*>(h);
  std::lock_guard<std::mutex> lock(s.mu);
  if (!s.dry) retire_completed(s);
  *live_events = s.live_events;
  if (ntasks) *ntasks = static_cast<int64_t>(s.tasks.size());
  return ok();
}

extern "C" jacc_status jacc_sched_join(jacc_sched h, uintptr_t stream) {
  if (!h) return fail(JACC_ERR_INVALID_ARG, "NULL scheduler");
  Sched& s = *reinterpret_cast<Sched*>(h);
  std::lock_guard<std::mutex> lock(s.mu);
  if (s.dry) return ok();
  for (size_t i = 0; i < s.streams.size(); ++i) {
    if (s.last_task[i] < 0) continue;
    const Task& t = s.tasks[s.last_task[i]];
    if (t.open) return fail(JACC_ERR_INVALID_ARG, "a nest task was not ended");
    jacc_status st =
        cuda_check(cudaStreamWaitEvent(reinterpret_cast<cudaStream_t>(stream), t.done, 0), "cudaStreamWaitEvent");
    if (st) return st;
  }
  return ok();
}

extern "C" jacc_status jacc_sched_release(jacc_sched h) {
  if (!h) return fail(JACC_ERR_INVALID_ARG, "NULL scheduler");
  Sched* s = reinterpret_cast<Sched*>(h);
  if (!s->dry) {
    for (cudaStream_t c : s->streams) cudaStreamSynchronize(c);
    for (Task& t : s->tasks)
      if (t.done) cudaEventDestroy(t.done);
    for (cudaStream_t c : s->streams) cudaStreamDestroy(c);
  }
  delete s;
  return ok();
}
