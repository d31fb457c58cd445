// Host-only check of the request loop's device-memory admission (csrc/admission.h): budget,
// session reuse, least-recently-used eviction, and that a request which cannot be admitted
// evicts nothing.  Exits non-zero on the first failed check.
#include <chrono>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "paper_2104_12282_gb300/csrc/admission.h"

using tomo_serve::Admission;
using tomo_serve::Clock;
using tomo_serve::Slot;

#define CHECK(cond)                                                      \
  do {                                                                   \
    if (!(cond)) {                                                       \
      std::printf("admission check failed at line %d: %s\n", __LINE__, #cond); \
      std::exit(1);                                                      \
    }                                                                    \
  } while (0)

static tomo_grid* fake_grid(int k) {
  return reinterpret_cast<tomo_grid*>(static_cast<uintptr_t>(0x1000) * (k + 1));
}

static tomo_grid_desc problem(int nx) {
  tomo_grid_desc d{};
  d.nx = nx;
  d.ny = nx / 2;
  d.nz = nx / 2;
  d.h = 1.0;
  d.E0 = 1.0;
  d.Emin = 1e-9;
  d.nu = 0.3;
  d.penal = 3.0;
  d.rmin = 1.5;
  d.precision = TOMO_FP32;
  d.precond = TOMO_PRECOND_MG;
  d.rtol = 1e-6;
  return d;
}

static Clock::time_point at(int ms) { return Clock::time_point() + std::chrono::milliseconds(ms); }

int main() {
  Admission A;
  A.budget = 100;
  std::vector<tomo_grid*> dead;
  const tomo_grid_desc d8 = problem(8), d16 = problem(16);

  // two requests fit side by side without eviction
  Slot* a = A.admit(0, d8, 40, dead);
  CHECK(a && a->busy && A.resident == 40);
  a->grid = fake_grid(0);
  Slot* b = A.admit(1, d8, 40, dead);
  CHECK(b && b != a && A.resident == 80 && dead.empty() && A.evictions == 0);
  b->grid = fake_grid(1);

  // a session whose grid is busy waits
  CHECK(A.admit(0, d8, 40, dead) == nullptr);

  // an idle session grid is reused for the same problem, with no new reservation
  A.release(a, true, at(1), dead);
  CHECK(!a->busy && dead.empty());
  CHECK(A.admit(0, d8, 40, dead) == a && a->busy && A.resident == 80);

  // the same session on another problem gets a new grid; the idle one is evicted for room
  A.release(a, true, at(2), dead);
  Slot* c = A.admit(0, d16, 40, dead);
  // (the evicted slot's memory may be reused for the new one: compare contents)
  CHECK(c && c->desc.nx == 16 && !c->grid && A.resident == 80 && A.evictions == 1);
  CHECK(A.slots.size() == 2);
  CHECK(dead.size() == 1 && dead[0] == fake_grid(0));
  dead.clear();
  c->grid = fake_grid(2);

  // busy grids hold the budget: the request waits
  CHECK(A.admit(2, d8, 40, dead) == nullptr && dead.empty() && A.evictions == 1);

  // evicting every idle grid would still not make room: nothing is evicted
  A.release(b, true, at(3), dead);
  CHECK(A.admit(3, d8, 70, dead) == nullptr);
  CHECK(dead.empty() && A.evictions == 1 && A.slots.size() == 2 && A.resident == 80);

  // with both grids idle, the least recently used goes first, then the next
  A.release(c, true, at(4), dead);
  Slot* e = A.admit(3, d8, 70, dead);
  CHECK(e && A.resident == 70 && A.evictions == 3 && A.slots.size() == 1);
  CHECK(dead.size() == 2 && dead[0] == fake_grid(1) && dead[1] == fake_grid(2));
  dead.clear();
  e->grid = fake_grid(3);

  // only what must go is evicted: room for a small request after a partial eviction
  Slot* f = A.admit(-1, d8, 30, dead);
  CHECK(f && A.resident == 100 && dead.empty());
  f->grid = fake_grid(4);
  A.release(e, true, at(5), dead);
  Slot* g = A.admit(5, d8, 20, dead);
  CHECK(g && A.resident == 50 && dead.size() == 1 && dead[0] == fake_grid(3));
  dead.clear();

  // a request with no session (or a failed one) frees its grid at once
  A.release(f, false, at(6), dead);
  CHECK(dead.size() == 1 && dead[0] == fake_grid(4) && A.resident == 20 && A.slots.size() == 1);
  dead.clear();
  A.release(g, false, at(7), dead);  // a grid never created: nothing to destroy
  CHECK(dead.empty() && A.resident == 0 && A.slots.empty());

  // a request larger than the whole budget is never admitted
  CHECK(A.admit(6, d8, 101, dead) == nullptr && A.slots.empty());

  // a session grid taking a request that needs more than it reserved (an optimisation run
  // on a grid made by a gradient request) reserves the difference, evicting other idle
  // grids for it but never itself; when even that cannot make room the request waits
  {
    Admission B;
    B.budget = 100;
    Slot* s0 = B.admit(0, d8, 40, dead);
    s0->grid = fake_grid(10);
    Slot* s1 = B.admit(1, d8, 40, dead);
    s1->grid = fake_grid(11);
    B.release(s1, true, at(10), dead);
    B.release(s0, true, at(11), dead);
    Slot* r = B.admit(0, d8, 70, dead);  // +30: evicts session 1's idle grid (LRU), not s0
    CHECK(r == s0 && r->busy && r->bytes == 70 && B.resident == 70);
    CHECK(dead.size() == 1 && dead[0] == fake_grid(11) && B.evictions == 1);
    dead.clear();
    B.release(r, true, at(12), dead);
    CHECK(B.admit(0, d8, 50, dead) == s0 && s0->bytes == 70 && B.resident == 70);  // fits
    B.release(s0, true, at(13), dead);
    Slot* o = B.admit(2, d8, 30, dead);
    CHECK(o && B.resident == 100);
    CHECK(B.admit(0, d8, 80, dead) == nullptr);  // +10 with only itself idle: waits
    CHECK(dead.empty() && s0->bytes == 70 && !s0->busy && B.resident == 100);
  }

  // problems that differ in any solver parameter are different problems
  tomo_grid_desc d8b = d8;
  d8b.rtol = 1e-8;
  CHECK(tomo_serve::same_problem(d8, d8) && !tomo_serve::same_problem(d8, d8b));
  CHECK(!tomo_serve::same_problem(d8, d16));

  std::printf("admission ok\n");
  return 0;
}
