// Host-side data parallelism for the graph build: contiguous index ranges
// handed out to up to 16 threads. Every user writes disjoint outputs per
// index (or combines per-range results with integer adds), so the result does
// not depend on the number of threads or on their timing.
#pragma once

#include <algorithm>
#include <atomic>
#include <cstdint>
#include <system_error>
#include <thread>
#include <vector>

namespace isingx {

inline int32_t host_threads() {
  const unsigned hw = std::thread::hardware_concurrency();
  return static_cast<int32_t>(std::max(1u, std::min(hw == 0 ? 1u : hw, 16u)));
}

// fn(lo, hi) over [0, count) in blocks of at least `grain` indices. Runs on
// the calling thread alone when count < 2 * grain, with one hardware thread,
// or when no thread can be started.
template <typename Fn>
void parallel_ranges(int64_t count, int64_t grain, Fn fn) {
  if (count <= 0) return;
  int32_t threads = host_threads();
  if (grain < 1) grain = 1;
  if (count < 2 * grain || threads <= 1) {
    fn(int64_t(0), count);
    return;
  }
  const int64_t nblocks = std::min<int64_t>((count + grain - 1) / grain, int64_t(threads) * 32);
  const int64_t block = (count + nblocks - 1) / nblocks;
  threads = static_cast<int32_t>(std::min<int64_t>(threads, nblocks));
  std::atomic<int64_t> next(0);
  auto work = [&] {
    for (int64_t b = next.fetch_add(1); b < nblocks; b = next.fetch_add(1)) {
      const int64_t lo = b * block, hi = std::min(count, lo + block);
      if (lo < hi) fn(lo, hi);
    }
  };
  std::vector<std::thread> pool;
  try {
    pool.reserve(static_cast<size_t>(threads));
    for (int32_t t = 1; t < threads; ++t) pool.emplace_back(work);
  } catch (const std::system_error&) {
    // fewer helpers: the blocks they would have taken go to the others
  } catch (const std::bad_alloc&) {
  }
  work();
  for (std::thread& t : pool) t.join();
}

// fn(lo, hi) over the rows [0, rows) of a CSR whose row r holds entries
// [off[r], off[r + 1]), in blocks of about equal entry counts (a row longer
// than a block's share forms a block of its own), so that a few long rows do
// not leave one thread with most of the work.
template <typename Off, typename Fn>
void parallel_rows(int64_t rows, const Off* off, Fn fn) {
  if (rows <= 0) return;
  const int64_t entries = static_cast<int64_t>(off[rows]) - static_cast<int64_t>(off[0]);
  const int64_t nblocks = std::min<int64_t>(int64_t(host_threads()) * 32, rows);
  if (nblocks <= 1 || entries + rows < (int64_t(1) << 19)) {
    fn(int64_t(0), rows);
    return;
  }
  // block b starts at the first row whose cost (entries before it plus one
  // per row) reaches b / nblocks of the total
  const int64_t total = entries + rows;
  std::vector<int64_t> start(static_cast<size_t>(nblocks) + 1, rows);
  start[0] = 0;
  for (int64_t b = 1; b < nblocks; ++b) {
    const int64_t target = total * b / nblocks;
    int64_t lo = start[static_cast<size_t>(b) - 1], hi = rows;
    while (lo < hi) {  // first r with off[r] - off[0] + r >= target
      const int64_t mid = lo + (hi - lo) / 2;
      if (static_cast<int64_t>(off[mid]) - static_cast<int64_t>(off[0]) + mid >= target)
        hi = mid;
      else
        lo = mid + 1;
    }
    start[static_cast<size_t>(b)] = lo;
  }
  parallel_ranges(nblocks, 1, [&](int64_t b0, int64_t b1) {
    for (int64_t b = b0; b < b1; ++b) {
      const int64_t lo = start[static_cast<size_t>(b)], hi = start[static_cast<size_t>(b) + 1];
      if (lo < hi) fn(lo, hi);
    }
  });
}

}  // namespace isingx
