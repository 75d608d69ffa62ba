// Host-side checks of the library's internal helpers (compiled and run by
// test_host_helpers_cpu.py): the byte-range overlap test that the entry points
// use to reject aliased vectors, and the graph-cache key, which must keep every
// (method tag, preconditioner) variant of a solve apart, also for right-hand
// sides one element apart.
#include <cstdio>
#include <set>
#include <tuple>

#include "internal.hpp"

static int failures = 0;
#define CHECK(c)                                              \
  do {                                                        \
    if (!(c)) {                                               \
      std::printf("FAILED line %d: %s\n", __LINE__, #c);      \
      ++failures;                                             \
    }                                                         \
  } while (0)

int main() {
  alignas(16) static char buf[1024];
  char* b = buf;
  // overlaps: half-open byte ranges
  CHECK(!helm::overlaps(b, 16, b + 16, 16));  // adjacent
  CHECK(!helm::overlaps(b + 16, 16, b, 16));
  CHECK(helm::overlaps(b, 16, b + 15, 16));   // one shared byte
  CHECK(helm::overlaps(b + 15, 16, b, 16));
  CHECK(helm::overlaps(b, 64, b, 64));        // identical
  CHECK(helm::overlaps(b, 256, b + 64, 16));  // one inside the other
  CHECK(helm::overlaps(b + 64, 16, b, 256));
  CHECK(!helm::overlaps(b, 0, b, 16));        // empty ranges share nothing
  CHECK(!helm::overlaps(b, 16, b, 0));
  CHECK(!helm::overlaps(b, 16, b + 512, 16));
  // graph keys: every (tag, preconditioner) variant on b, and on b + 16 bytes,
  // with one x, are distinct
  helm_opts none, jac;
  none.precond = HELM_PRECOND_NONE;
  jac.precond = HELM_PRECOND_JACOBI;
  std::set<std::tuple<const void*, const void*, int>> keys;
  int made = 0;
  for (int shift = 0; shift <= 32; shift += 16)
    for (int tag = 0; tag <= 12; ++tag)
      for (const helm_opts* o : {&none, &jac}) {
        keys.insert(helm::graph_key(b + shift, b + 512, tag, *o));
        ++made;
      }
  CHECK(static_cast<int>(keys.size()) == made);
  CHECK(helm::graph_key(b, b + 512, 0, jac) != helm::graph_key(b + 16, b + 512, 0, none));
  CHECK(helm::graph_key(b, b + 512, 3, none) == helm::graph_key(b, b + 512, 3, none));
  if (failures == 0) std::printf("ok\n");
  return failures == 0 ? 0 : 1;
}
