// Host-side parallel loops for mesh preparation and the multigrid setup.
//
// Work is cut into chunks whose bounds depend only on the problem size, never
// on the number of threads; a body writes only what its chunk owns, and every
// reduction combines chunk results in chunk order.  Results are therefore bit
// for bit the same for any thread count, including one.
#pragma once

#include <algorithm>
#include <cstdint>
#include <functional>

namespace ifilt {

// Worker threads for host loops: IFILT_HOST_THREADS if set (>= 1), else the
// hardware threads, at most 64.
int host_threads();

// Runs body(chunk, worker) for chunk = 0 .. n_chunks-1 on up to host_threads()
// threads (worker < host_threads() names a per-thread scratch slot).  The
// first exception a body throws is rethrown after every thread has stopped.
void parallel_chunks(int64_t n_chunks, const std::function<void(int64_t chunk, int worker)>& body);

// Chunks of `chunk` consecutive indices over [0, n): body(begin, end, worker).
inline void parallel_range(int64_t n, int64_t chunk, const std::function<void(int64_t, int64_t, int)>& body) {
  if (n <= 0) return;
  const int64_t nc = (n + chunk - 1) / chunk;
  parallel_chunks(nc, [&](int64_t c, int w) { body(c * chunk, std::min(n, (c + 1) * chunk), w); });
}

// Stable insertion sort of a short run (used per sparse row, where runs hold
// tens of entries); longer runs fall back to std::stable_sort.
template <typename T, typename Less>
void stable_sort_small(T* a, int64_t n, Less less) {
  if (n > 48) {
    std::stable_sort(a, a + n, less);
    return;
  }
  for (int64_t i = 1; i < n; i++) {
    T x = a[i];
    int64_t j = i;
    while (j > 0 && less(x, a[j - 1])) {
      a[j] = a[j - 1];
      j--;
    }
    a[j] = x;
  }
}

}  // namespace ifilt
