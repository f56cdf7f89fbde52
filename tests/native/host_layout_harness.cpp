// Host build of the host-memory solve's workspace layout
// (paper_2107_05395_gb300/csrc/host_layout.h) for CPU unit tests
// (compiled by tests/test_host_layout.py).
#include "../../paper_2107_05395_gb300/csrc/host_layout.h"

extern "C" {
int h_slots() { return sb::kHostSlots; }
unsigned long h_slot_x_offset(long N, long C, unsigned long rs) { return sb::host_slot_x_offset(N, C, rs); }
unsigned long h_slot_bytes(long N, long C, unsigned long rs, unsigned long xs) {
  return sb::host_slot_bytes(N, C, rs, xs);
}
}
