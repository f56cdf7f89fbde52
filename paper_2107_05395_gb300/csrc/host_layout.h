// Layout of the device workspace of the host-memory solve (host_io.cpp): kHostSlots
// slots, each holding one chunk's right-hand sides followed by its solutions.  Each
// part starts on a 256-byte boundary, so an FP64 solution part that follows FP32
// right-hand sides of an odd element count is still aligned, and so is every slot.
// Plain C++ (no CUDA) so that the CPU tests compile it on its own.
#pragma once

#include <cstddef>
#include <cstdint>

namespace sb {

constexpr int kHostSlots = 3;

inline size_t host_round256(size_t b) { return (b + 255) / 256 * 256; }

// Byte offset of the solution part within a slot of C systems of N rows.
inline size_t host_slot_x_offset(int64_t N, int64_t C, size_t rhs_elem) {
  return host_round256((size_t)N * (size_t)C * rhs_elem);
}

// Bytes of one slot.
inline size_t host_slot_bytes(int64_t N, int64_t C, size_t rhs_elem, size_t x_elem) {
  return host_slot_x_offset(N, C, rhs_elem) + host_round256((size_t)N * (size_t)C * x_elem);
}

}  // namespace sb
