// bit3_layout.h -- shared-memory layout of the "bit3" policy (bit3.cuh),
// used by the host plan and the kernel alike.
#pragma once

namespace fr {

constexpr int kB3Warps = 8;           // warps (tiles in flight) per block
constexpr int kB3Pitch = 29;          // box rows per plane (27 + 2 halo)
constexpr int kB3BoxWords = 844;      // 29 x 29 rows, padded to 16 bytes
// per-warp shared memory: the box, 26 neighbour-tile pointers, the tile's
// result bits in omega order (k^3 bits)
constexpr int kB3OffPtr = 4 * kB3BoxWords;
constexpr int kB3OffBits = kB3OffPtr + 224;   // 27 pointers (the bit-state path indexes all 27 directions)

// Bit-packed state of a tile between generations of a multi-generation run:
// its 27 x 27 inner box rows (cells x = 0..26 at bits 1..27, row (y, z) at
// word (y - 1) + 27 (z - 1)), then its faces x = 0 and x = 26 as 27 words
// each (word z: bit y = cell (0 or 26, y, z)); padded to 16 bytes.
constexpr int kB3StateWords = 784;
constexpr int kB3StatePtrBytes = 224;         // per warp in generations from states to states: 27 pointers
constexpr int kB3StateXL = 729;
constexpr int kB3StateXH = 756;

}  // namespace fr
