// lb_sched.h -- admission policy of the serving form (host-only C++17, no
// CUDA): requests wait in arrival order and are admitted while a slot is free
// and their device-memory footprint fits in what the budget has left.  A
// request that does not fit lets later ones pass it only until it has waited
// `bypass_ms`; from then on it blocks the queue until memory frees up, so a
// large request cannot starve behind a stream of small ones.
#pragma once

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <deque>
#include <vector>

namespace lbs {

struct Pending {
  uint64_t id;
  int64_t bytes;
  double t_submit_ms;
};

struct Policy {
  int64_t budget = 0;
  int slots = 1;
  double bypass_ms = 0.0;
  int64_t used = 0;
  int inflight = 0;

  bool fits(int64_t b) const { return inflight < slots && used + b <= budget; }

  // Admit from q at time now_ms; admitted requests leave q, their bytes are
  // charged and their ids returned in admission order.
  std::vector<uint64_t> admit(std::deque<Pending>& q, double now_ms) {
    std::vector<uint64_t> out;
    for (auto it = q.begin(); it != q.end() && inflight < slots;) {
      if (fits(it->bytes)) {
        used += it->bytes;
        ++inflight;
        out.push_back(it->id);
        it = q.erase(it);
      } else if (now_ms - it->t_submit_ms >= bypass_ms) {
        break;  // waited long enough: nobody behind it may pass
      } else {
        ++it;
      }
    }
    return out;
  }

  void release(int64_t b) {
    used -= b;
    --inflight;
  }
};

// Nearest-rank percentile (q in [0, 100]) of x; 0 for an empty sample.
inline double percentile(std::vector<double> x, double q) {
  if (x.empty()) return 0.0;
  std::sort(x.begin(), x.end());
  const double n = (double)x.size();
  int64_t k = (int64_t)std::ceil(q / 100.0 * n) - 1;
  k = std::max<int64_t>(0, std::min<int64_t>(k, (int64_t)x.size() - 1));
  return x[(size_t)k];
}

// Discrete-event replay of the policy: request i arrives at arrival[i] (ms,
// non-decreasing), holds bytes[i] and runs service[i] ms once admitted,
// independently of the others.  Admission runs after every arrival and
// completion.  start/finish receive the times (-1 for a request larger than
// the budget, which is never admitted).
inline void simulate(int n, const double* arrival, const int64_t* bytes, const double* service, int64_t budget,
                     int slots, double bypass_ms, double* start, double* finish) {
  Policy pol;
  pol.budget = budget;
  pol.slots = slots;
  pol.bypass_ms = bypass_ms;
  std::deque<Pending> q;
  struct Run {
    double t;
    int i;
  };
  std::vector<Run> running;
  int next = 0;
  for (int i = 0; i < n; ++i) start[i] = finish[i] = -1.0;
  while (next < n || !q.empty() || !running.empty()) {
    double t = 1e300;
    if (next < n) t = arrival[next];
    for (const Run& r : running) t = std::min(t, r.t);
    if (t == 1e300) break;  // only never-admissible requests are left
    for (size_t k = 0; k < running.size();) {
      if (running[k].t <= t) {
        pol.release(bytes[running[k].i]);
        running[k] = running.back();
        running.pop_back();
      } else {
        ++k;
      }
    }
    while (next < n && arrival[next] <= t) {
      if (bytes[next] <= budget) q.push_back(Pending{(uint64_t)next, bytes[next], arrival[next]});
      ++next;
    }
    for (uint64_t id : pol.admit(q, t)) {
      const int i = (int)id;
      start[i] = t;
      finish[i] = t + service[i];
      running.push_back(Run{finish[i], i});
    }
    if (next >= n && running.empty() && !q.empty()) break;  // cannot happen: an empty GPU admits the head
  }
}

}  // namespace lbs
