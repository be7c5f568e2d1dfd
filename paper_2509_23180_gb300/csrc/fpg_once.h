// Once-per-device host set-up (kernel attributes), safe under several host threads.
// Host code only: needs the CUDA runtime API declarations and the C++ library.
#pragma once

#include <cuda_runtime_api.h>

#include <atomic>
#include <mutex>
#include <utility>

namespace fpg {

// Function attributes (cudaFuncSetAttribute) apply to the current device only, so
// a kernel's attributes are set once per device, before its first launch there.
// Use as `if (auto once = x.first()) { ...set attributes... }`: the guard is true
// for the first caller on the current device (and always for device ordinals past
// 63) and holds the struct's lock until the end of that block; the device is marked
// done only when the block has run.  Host threads that arrive meanwhile wait on the
// lock, so none launches the kernel before its attributes are set.
struct PerDeviceOnce {
  std::mutex mu;
  std::atomic<bool> done[64] = {};
  class Guard {
   public:
    Guard() = default;
    Guard(Guard&& o) noexcept : owner_(o.owner_), dev_(o.dev_), first_(o.first_), lk_(std::move(o.lk_)) {
      o.owner_ = nullptr;
    }
    Guard(const Guard&) = delete;
    Guard& operator=(const Guard&) = delete;
    Guard& operator=(Guard&&) = delete;
    ~Guard() {  // marks the device done, then releases the lock (member destruction)
      if (owner_ != nullptr && dev_ >= 0) owner_->done[dev_].store(true, std::memory_order_release);
    }
    explicit operator bool() const { return first_; }

   private:
    friend struct PerDeviceOnce;
    PerDeviceOnce* owner_ = nullptr;
    int dev_ = -1;
    bool first_ = false;
    std::unique_lock<std::mutex> lk_;
  };
  Guard first() {
    Guard g;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
      g.first_ = true;  // no per-device record: set the attributes every time
      return g;
    }
    if (done[dev].load(std::memory_order_acquire)) return g;
    g.lk_ = std::unique_lock<std::mutex>(mu);
    if (done[dev].load(std::memory_order_relaxed)) {
      g.lk_.unlock();
      return g;
    }
    g.owner_ = this;
    g.dev_ = dev;
    g.first_ = true;
    return g;
  }
};

}  // namespace fpg
