// rows_layout.h -- compile-time unit layout of the "rows" policy of the
// compact step, for 2D fractals with s = 3 whose level-1 pattern is known at
// compile time (the Sierpinski carpet F^{8,3} and the Vicsek fractal
// F^{5,3}, Table 1, offsets numbered row-major over the 3x3 digit box).
//
// A thread owns a unit: the k^2 cells of one level-2 subtree (consecutive in
// omega order), which fill the unit's 9x9 block in the embedding.  It builds
// the block's 9 rows, plus the frame of the 11x11 window around it (the cells
// of the 8 neighbouring units that touch the block), as byte rows of three
// words (columns -1..10), sums every 3x3 window with byte-wise SWAR
// (vertical sum of three rows, then of three shifted copies; sums <= 9 never
// carry across bytes), gathers the totals back into omega order and applies
// the rule to 4 cells at once.  Which byte of which word each row byte and
// each omega byte comes from follows from the level-1 pattern; this header
// works it out at compile time (rows.cuh turns it into prmt selectors), and
// the host plan uses the same functions for the neighbour-unit tables.
#pragma once

#include <stdint.h>

namespace fr {

template <int P>
struct RowsPreset;
template <>
struct RowsPreset<0> {   // carpet: the 3x3 digit box without its centre
    static constexpr int k = 8;
    static constexpr int ox[8] = {0, 1, 2, 0, 2, 0, 1, 2};
    static constexpr int oy[8] = {0, 0, 0, 1, 1, 2, 2, 2};
};
template <>
struct RowsPreset<1> {   // Vicsek: the centre and its 4 orthogonal neighbours
    static constexpr int k = 5;
    static constexpr int ox[5] = {1, 0, 1, 2, 1};
    static constexpr int oy[5] = {0, 1, 1, 1, 2};
};

// replica at digit tuple (x1, y1), -1 none
template <int P>
constexpr int rp_id(int x1, int y1)
{
    for (int j = 0; j < RowsPreset<P>::k; ++j)
        if (RowsPreset<P>::ox[j] == x1 && RowsPreset<P>::oy[j] == y1) return j;
    return -1;
}

// byte of the unit (omega order within it) of the cell at (x, y) of the
// unit's 9x9 block, -1 for a hole
template <int P>
constexpr int rp_byte(int x, int y)
{
    if (x < 0 || x > 8 || y < 0 || y > 8) return -1;
    const int j = rp_id<P>(x / 3, y / 3), l = rp_id<P>(x % 3, y % 3);
    return (j < 0 || l < 0) ? -1 : RowsPreset<P>::k * j + l;
}

// Byte offset of unit slot n in a stage.  The carpet's 64-byte units sit in
// groups of rp_group consecutive units with a 16-byte gap after each group,
// so that one bulk copy brings a whole group and the 16-byte loads of the
// units a quarter-warp handles (rp_thread_unit) hit 8 different bank groups
// (at a plain 64-byte stride every unit would start in one of 2 of them).
// The Vicsek fractal's 25-byte units stay contiguous.
template <int P>
constexpr bool rp_padded()
{
    return P == 0;
}
template <int P>
constexpr int rp_group()
{
    return rp_padded<P>() ? 8 : 1;
}
template <int P>
constexpr int rp_slot(int n)
{
    return rp_padded<P>() ? (64 * rp_group<P>() + 16) * (n / rp_group<P>()) + 64 * (n % rp_group<P>())
                          : RowsPreset<P>::k * RowsPreset<P>::k * n;
}
// The unit thread q handles in a tile of nq units.  For padded units and
// whole warps of units, lane l of warp w takes unit 32 w + 8 g + 2 h + b
// with g = (l & 7) >> 1, h = l >> 3, b = l & 1: the 8 lanes of quarter-warp
// h read from groups g = 0..3 (offsets 16 g mod 128, the group stride being
// 16 more than 4 x 128) at units 2 h + b of each (64 b mod 128), that is 8
// distinct 16-byte bank groups.  Otherwise the identity.
template <int P>
constexpr int rp_thread_unit(int q, int nq)
{
    if (rp_group<P>() != 8 || (nq & 31)) return q;
    const int l = q & 31;
    return (q & ~31) + 8 * ((l & 7) >> 1) + 2 * (l >> 3) + (l & 1);
}

template <int P>
constexpr int rp_x(int u)
{
    return 3 * RowsPreset<P>::ox[u / RowsPreset<P>::k] + RowsPreset<P>::ox[u % RowsPreset<P>::k];
}
template <int P>
constexpr int rp_y(int u)
{
    return 3 * RowsPreset<P>::oy[u / RowsPreset<P>::k] + RowsPreset<P>::oy[u % RowsPreset<P>::k];
}

// The frame of the unit's 11x11 window: 40 positions t, top row (x = -1..9,
// y = -1), bottom row (y = 9), left column (x = -1, y = 0..8), right column.
constexpr int kFrame = 40;
constexpr int frame_x(int t) { return t < 11 ? t - 1 : (t < 22 ? t - 12 : (t < 31 ? -1 : 9)); }
constexpr int frame_y(int t) { return t < 11 ? -1 : (t < 22 ? 9 : (t < 31 ? t - 22 : t - 31)); }
constexpr int frame_at(int x, int y)
{
    for (int t = 0; t < kFrame; ++t)
        if (frame_x(t) == x && frame_y(t) == y) return t;
    return -1;
}
// neighbouring unit of frame position t: direction slot 0..7 (W..E, N..S
// row-major over (dx, dy) without the centre) and the byte of that unit
constexpr int frame_dir(int t)
{
    const int x = frame_x(t), y = frame_y(t);
    const int dx = x < 0 ? -1 : (x > 8 ? 1 : 0), dy = y < 0 ? -1 : (y > 8 ? 1 : 0);
    const int d9 = (dx + 1) + 3 * (dy + 1);
    return d9 < 4 ? d9 : d9 - 1;
}
template <int P>
constexpr int frame_byte(int t)
{
    return rp_byte<P>((frame_x(t) + 9) % 9, (frame_y(t) + 9) % 9);
}
// external cells: the frame positions that are members, numbered e
template <int P>
constexpr int rp_next()
{
    int n = 0;
    for (int t = 0; t < kFrame; ++t) n += frame_byte<P>(t) >= 0;
    return n;
}
template <int P>
constexpr int ext_of_frame(int t)
{
    if (frame_byte<P>(t) < 0) return -1;
    int e = 0;
    for (int u = 0; u < t; ++u) e += frame_byte<P>(u) >= 0;
    return e;
}
template <int P>
constexpr int frame_of_ext(int e)
{
    for (int t = 0; t < kFrame; ++t)
        if (ext_of_frame<P>(t) == e) return t;
    return -1;
}

}  // namespace fr
