// Host-side passes over a request's arrays (validation, diagonal sums, copies) on several
// threads.  A large CSR request (tens of millions of entries) otherwise spends hundreds of
// milliseconds of one core in these passes, inside the caller's submit or create call.
//
// The work is cut into chunks whose boundaries depend only on the array sizes, never on
// the number of threads, and per-chunk partial results are combined in chunk order: the
// results are the same on every machine.
#pragma once
#include <algorithm>
#include <atomic>
#include <cstring>
#include <thread>
#include <vector>

namespace pcgk {
namespace host {

constexpr int kMaxThreads = 16;
constexpr long long kRowsPerChunk = 1LL << 16;     // validation and diagonal passes
constexpr size_t kCopyChunkBytes = size_t(8) << 20;  // copies

// Runs fn(c) for every chunk c in [0, nchunks), on up to kMaxThreads threads (the caller's
// included).  A thread that cannot be started leaves its share to the others.
template <class F>
void for_chunks(long long nchunks, F&& fn) {
  if (nchunks <= 0) return;
  const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
  const int T = (int)std::min<long long>({nchunks, (long long)hw, (long long)kMaxThreads});
  if (T <= 1) {
    for (long long c = 0; c < nchunks; ++c) fn(c);
    return;
  }
  std::atomic<long long> next{0};
  auto work = [&] {
    for (long long c = next.fetch_add(1); c < nchunks; c = next.fetch_add(1)) fn(c);
  };
  std::vector<std::thread> pool;
  pool.reserve(T - 1);
  for (int t = 1; t < T; ++t) {
    try {
      pool.emplace_back(work);
    } catch (...) {
      break;
    }
  }
  work();
  for (std::thread& t : pool) t.join();
}

// memcpy of `bytes` bytes in chunks on several threads.
inline void copy(void* dst, const void* src, size_t bytes) {
  if (bytes <= kCopyChunkBytes) {
    if (bytes) std::memcpy(dst, src, bytes);
    return;
  }
  const long long nc = (long long)((bytes + kCopyChunkBytes - 1) / kCopyChunkBytes);
  for_chunks(nc, [&](long long c) {
    const size_t off = (size_t)c * kCopyChunkBytes;
    std::memcpy((char*)dst + off, (const char*)src + off, std::min(kCopyChunkBytes, bytes - off));
  });
}

inline long long row_chunks(long long n) { return (n + kRowsPerChunk - 1) / kRowsPerChunk; }

// A vector allocator that leaves new elements uninitialised (they are copied into at once;
// zero-filling first would be one more pass over memory).
template <class T>
struct UninitAlloc : std::allocator<T> {
  using value_type = T;
  template <class U>
  struct rebind {
    using other = UninitAlloc<U>;
  };
  UninitAlloc() = default;
  template <class U>
  UninitAlloc(const UninitAlloc<U>&) {}
  template <class U>
  void construct(U* p) noexcept {
    ::new ((void*)p) U;
  }
  template <class U, class... A>
  void construct(U* p, A&&... a) {
    ::new ((void*)p) U(std::forward<A>(a)...);
  }
};

template <class T>
using buffer = std::vector<T, UninitAlloc<T>>;

// dst = a copy of src[0 .. count).
template <class T>
void assign(buffer<T>& dst, const T* src, size_t count) {
  dst.resize(count);
  copy(dst.data(), src, count * sizeof(T));
}

}  // namespace host
}  // namespace pcgk
