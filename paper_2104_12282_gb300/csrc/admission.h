// Device-memory admission for the request loop (host only, no CUDA): the resident grids
// (slots) with the bytes each one reserves, a budget, and least-recently-used eviction of
// idle grids.  The caller serialises every call (the request loop holds its mutex).
//
// A request is admitted onto the idle resident grid of its session when that grid was made
// for the same problem (raising the slot's reservation when the request needs more than the
// grid reserved), or onto a new slot, when the bytes it adds fit the budget after evicting
// other idle grids, oldest use first.  Nothing is evicted unless the request is
// admitted: when busy grids hold too much of the budget the request waits and every idle
// grid stays resident.
#pragma once

#include <algorithm>
#include <chrono>
#include <cstddef>
#include <cstdint>
#include <memory>
#include <vector>

#include "../../include/tomo.h"

namespace tomo_serve {

using Clock = std::chrono::steady_clock;

struct Slot {
  tomo_grid* grid = nullptr;
  int64_t session = -1;
  tomo_grid_desc desc{};  // dims and parameters the grid was created with
  size_t bytes = 0;       // reserved (estimated) device bytes
  bool busy = false;
  Clock::time_point last_used;
};

inline bool same_problem(const tomo_grid_desc& a, const tomo_grid_desc& b) {
  return a.nx == b.nx && a.ny == b.ny && a.nz == b.nz && a.h == b.h && a.E0 == b.E0 &&
         a.Emin == b.Emin && a.nu == b.nu && a.penal == b.penal && a.rmin == b.rmin &&
         a.precision == b.precision && a.precond == b.precond && a.rtol == b.rtol &&
         a.maxit == b.maxit && a.mg_levels == b.mg_levels &&
         a.smoother_degree == b.smoother_degree && a.coarse_degree == b.coarse_degree &&
         a.cheb_ratio == b.cheb_ratio && a.cheb_lmax == b.cheb_lmax && a.rr_every == b.rr_every;
}

struct Admission {
  size_t budget = 0;
  size_t resident = 0;  // bytes reserved by all slots
  uint64_t evictions = 0;
  std::vector<std::unique_ptr<Slot>> slots;

  // The slot a request of `session` (-1: none) on problem `desc` needing `est` bytes runs
  // on, marked busy, or nullptr if it must wait.  Grids of evicted slots go into `dead`
  // (the caller destroys them outside its lock).
  Slot* admit(int64_t session, const tomo_grid_desc& desc, size_t est,
              std::vector<tomo_grid*>& dead) {
    Slot* reuse = nullptr;
    if (session >= 0)
      for (auto& s : slots)
        if (s->session == session && same_problem(s->desc, desc)) {
          if (s->busy) return nullptr;  // the session's grid is in use (or being created)
          reuse = s.get();
          break;
        }
    // bytes to reserve on top of what the slot holds: a resident grid may take a request
    // that needs more than it was created for (an optimisation run's design buffers)
    const size_t need = reuse ? (est > reuse->bytes ? est - reuse->bytes : 0) : est;
    size_t idle = 0;
    for (auto& s : slots)
      if (!s->busy && s.get() != reuse) idle += s->bytes;
    if (resident + need > budget + idle) return nullptr;  // busy grids hold the rest
    while (resident + need > budget) {
      Slot* lru = nullptr;
      for (auto& s : slots)
        if (!s->busy && s.get() != reuse && (!lru || s->last_used < lru->last_used))
          lru = s.get();
      if (!lru) return nullptr;  // unreachable: the check above leaves enough idle bytes
      resident -= lru->bytes;
      if (lru->grid) dead.push_back(lru->grid);
      evictions += 1;
      erase(lru);
    }
    resident += need;
    if (reuse) {
      reuse->bytes += need;
      reuse->busy = true;
      return reuse;
    }
    auto s = std::make_unique<Slot>();
    s->session = session;
    s->desc = desc;
    s->bytes = est;
    s->busy = true;
    slots.push_back(std::move(s));
    return slots.back().get();
  }

  // The request on `s` finished at `t`.  keep: the grid stays resident, idle, for the next
  // request of its session; otherwise the slot is freed now and its grid goes into `dead`.
  void release(Slot* s, bool keep, Clock::time_point t, std::vector<tomo_grid*>& dead) {
    s->busy = false;
    s->last_used = t;
    if (keep) return;
    if (s->grid) dead.push_back(s->grid);
    resident -= s->bytes;
    erase(s);
  }

 private:
  void erase(Slot* p) {
    slots.erase(std::find_if(slots.begin(), slots.end(),
                             [&](const std::unique_ptr<Slot>& q) { return q.get() == p; }));
  }
};

}  // namespace tomo_serve
