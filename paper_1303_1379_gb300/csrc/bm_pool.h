// Device-memory pool bookkeeping of the matching server: offsets into one
// cudaMalloc'd pool, no device calls (host code only; unit-tested on the CPU).
#pragma once

#include <cstddef>
#include <iterator>
#include <map>

namespace bms {

// First-fit allocator over [0, size) in 256-byte units, coalescing on free.
class PoolAllocator {
  public:
    explicit PoolAllocator(std::size_t size) : size_(size & ~std::size_t(255)) {
        if (size_) free_[0] = size_;
    }
    bool alloc(std::size_t bytes, std::size_t* off) {
        bytes = (bytes + 255) & ~std::size_t(255);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= bytes) {
                *off = it->first;
                const std::size_t rest = it->second - bytes, at = it->first + bytes;
                free_.erase(it);
                if (rest) free_[at] = rest;
                used_ += bytes;
                return true;
            }
        }
        return false;
    }
    void release(std::size_t off, std::size_t bytes) {
        bytes = (bytes + 255) & ~std::size_t(255);
        used_ -= bytes;
        auto it = free_.emplace(off, bytes).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
    std::size_t size() const { return size_; }
    std::size_t used() const { return used_; }

  private:
    std::size_t size_;
    std::size_t used_ = 0;
    std::map<std::size_t, std::size_t> free_;
};

}  // namespace bms
