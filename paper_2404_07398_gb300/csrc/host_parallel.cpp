// Host worker threads for preparation loops (see host_parallel.h).
#include "host_parallel.h"

#include <atomic>
#include <cstdlib>
#include <exception>
#include <mutex>
#include <thread>
#include <vector>

namespace ifilt {

int host_threads() {
  if (const char* e = std::getenv("IFILT_HOST_THREADS")) {
    const int v = std::atoi(e);
    if (v >= 1) return std::min(v, 64);
  }
  const unsigned hw = std::thread::hardware_concurrency();
  return (int)std::max(1u, std::min(hw, 64u));
}

void parallel_chunks(int64_t n_chunks, const std::function<void(int64_t, int)>& body) {
  if (n_chunks <= 0) return;
  const int nt = (int)std::min<int64_t>(host_threads(), n_chunks);
  if (nt <= 1) {
    for (int64_t c = 0; c < n_chunks; c++) body(c, 0);
    return;
  }
  std::atomic<int64_t> next{0};
  std::atomic<bool> stop{false};
  std::exception_ptr err;
  std::mutex err_mu;
  auto run = [&](int w) {
    for (;;) {
      if (stop.load(std::memory_order_relaxed)) return;
      const int64_t c = next.fetch_add(1, std::memory_order_relaxed);
      if (c >= n_chunks) return;
      try {
        body(c, w);
      } catch (...) {
        std::lock_guard<std::mutex> lk(err_mu);
        if (!err) err = std::current_exception();
        stop.store(true);
        return;
      }
    }
  };
  std::vector<std::thread> th;
  th.reserve((size_t)nt - 1);
  try {
    for (int w = 1; w < nt; w++) th.emplace_back(run, w);
  } catch (...) {
    // could not start every thread: the ones that started and this one finish the work
  }
  run(0);
  for (auto& t : th) t.join();
  if (err) std::rethrow_exception(err);
}

}  // namespace ifilt
