// Bits of the device status word of a call (0 = ok), read back at the end of
// the call and reported as FPT_EDEVICE_STATUS.
#pragma once

namespace fpt {

constexpr unsigned kStatusWaitExpired = 1u;   // a bounded tensor-core wait gave up
// set only by the bounds checks of an FPT_DEBUG build, which then skip the access:
constexpr unsigned kStatusSetIndex = 0x10u;   // a ticket's parameter set does not hold its record
constexpr unsigned kStatusQueueFull = 0x20u;  // a warp's replay queue would overflow
constexpr unsigned kStatusRecord = 0x40u;     // a record index at or beyond the run total
constexpr unsigned kStatusHistBin = 0x80u;    // a histogram bin index beyond the edge clamp

}  // namespace fpt

// FPT_DEBUG=1 builds the bounds checks into the kernels (a separate library,
// paper_2206_11234_gb300/libfpt_gb300_debug.so); the default build has none.
#ifndef FPT_DEBUG
#define FPT_DEBUG 0
#endif
