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
constexpr int kB3OffBits = kB3OffPtr + 208;

}  // namespace fr
