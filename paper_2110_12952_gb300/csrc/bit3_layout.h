// bit3_layout.h -- shared-memory layout and halo-row order of the "bit3"
// policy (bit3.cuh), used by the host plan and the kernel alike.
#pragma once

namespace fr {

constexpr int kB3Warps = 8;           // warps (tiles in flight) per block
constexpr int kB3Pitch = 29;          // box rows per plane (27 + 2 halo)
constexpr int kB3BoxWords = 844;      // 29 x 29 rows, padded to 16 bytes
constexpr int kB3IoBytes = 768;       // 32 blocks of at most 24 cells
constexpr int kB3WarpBytes = 4 * kB3BoxWords + kB3IoBytes;
constexpr int kB3FullRows = 112;      // rows with y or z on the halo
constexpr int kB3Inner = 729;         // the other rows

// Box row (y + 29 z) of the i-th row with y or z on the halo: the plane
// z = 0, the plane z = 28, then rows y = 0 and y = 28 of each inner plane.
__host__ __device__ __forceinline__ int b3_full_row(int i)
{
    if (i < 29) return i;
    if (i < 58) return (i - 29) + kB3Pitch * 28;
    const int j = i - 58;
    return (j & 1) * 28 + kB3Pitch * (1 + (j >> 1));
}

}  // namespace fr
