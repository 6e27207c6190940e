// lid_layout.h -- compile-time unit layout of the "lid" policy of the
// compact step: the 3x3 sums of the cells of a unit (the k^U cells of a
// level-U subtree, consecutive in omega order) written directly in omega
// order, as a sum over the 9 directions of byte permutations of the unit's
// own bytes (plus the few cells of neighbouring units that touch it).  For
// a fractal whose members touch few other members (the Vicsek fractal: at
// most 4) this needs no 2D rows at all.  The host plan uses the same
// functions for the neighbour-unit tables.
#pragma once

#include <stdint.h>

#include "rows_layout.h"

namespace fr {

constexpr int cpow(int b, int e)
{
    int v = 1;
    for (int i = 0; i < e; ++i) v *= b;
    return v;
}

template <int P, int U>
struct LidUnit {
    static constexpr int k = RowsPreset<P>::k;
    static constexpr int side = cpow(3, U);   // the unit's block is side x side
    static constexpr int NB = cpow(k, U);     // cells (bytes) per unit
};

// position of byte u of the unit in its block
template <int P, int U>
constexpr int lu_x(int u)
{
    int x = 0, sc = 1;
    for (int m = 0; m < U; ++m, sc *= 3, u /= RowsPreset<P>::k) x += sc * RowsPreset<P>::ox[u % RowsPreset<P>::k];
    return x;
}
template <int P, int U>
constexpr int lu_y(int u)
{
    int y = 0, sc = 1;
    for (int m = 0; m < U; ++m, sc *= 3, u /= RowsPreset<P>::k) y += sc * RowsPreset<P>::oy[u % RowsPreset<P>::k];
    return y;
}
// byte of the cell at (x, y) of the unit's block, -1 for a hole
template <int P, int U>
constexpr int lu_byte(int x, int y)
{
    if (x < 0 || y < 0 || x >= LidUnit<P, U>::side || y >= LidUnit<P, U>::side) return -1;
    int u = 0, kp = 1;
    for (int m = 0; m < U; ++m, kp *= RowsPreset<P>::k, x /= 3, y /= 3) {
        const int j = rp_id<P>(x % 3, y % 3);
        if (j < 0) return -1;
        u += kp * j;
    }
    return u;
}

// The frame of the unit's window: the positions just outside its block.
// Frame position (x, y) lies in the neighbouring unit of direction slot
// lu_dir (0..7, (dx, dy) row-major without the centre) at byte lu_fbyte.
template <int P, int U>
constexpr int lu_dir(int x, int y)
{
    constexpr int S = LidUnit<P, U>::side;
    const int dx = x < 0 ? -1 : (x >= S ? 1 : 0), dy = y < 0 ? -1 : (y >= S ? 1 : 0);
    const int d9 = (dx + 1) + 3 * (dy + 1);
    return d9 < 4 ? d9 : d9 - 1;
}
template <int P, int U>
constexpr int lu_fbyte(int x, int y)
{
    constexpr int S = LidUnit<P, U>::side;
    return lu_byte<P, U>((x + S) % S, (y + S) % S);
}
// external cells: frame positions that are members and touch a member of
// the unit, numbered e in scan order of the frame (y, then x)
template <int P, int U>
constexpr bool lu_is_ext(int x, int y)
{
    constexpr int S = LidUnit<P, U>::side;
    const bool frame = (x == -1 || x == S || y == -1 || y == S) && x >= -1 && x <= S && y >= -1 && y <= S;
    if (!frame || lu_fbyte<P, U>(x, y) < 0) return false;
    for (int dy = -1; dy <= 1; ++dy)
        for (int dx = -1; dx <= 1; ++dx)
            if (lu_byte<P, U>(x + dx, y + dy) >= 0) return true;
    return false;
}
template <int P, int U>
constexpr int lu_next()
{
    constexpr int S = LidUnit<P, U>::side;
    int n = 0;
    for (int y = -1; y <= S; ++y)
        for (int x = -1; x <= S; ++x) n += lu_is_ext<P, U>(x, y);
    return n;
}
template <int P, int U>
constexpr int lu_ext_index(int x, int y)
{
    constexpr int S = LidUnit<P, U>::side;
    if (!lu_is_ext<P, U>(x, y)) return -1;
    int n = 0;
    for (int yy = -1; yy <= S; ++yy)
        for (int xx = -1; xx <= S; ++xx) {
            if (xx == x && yy == y) return n;
            n += lu_is_ext<P, U>(xx, yy);
        }
    return -1;
}
template <int P, int U>
constexpr int lu_ext_x(int e)
{
    constexpr int S = LidUnit<P, U>::side;
    for (int y = -1; y <= S; ++y)
        for (int x = -1; x <= S; ++x)
            if (lu_ext_index<P, U>(x, y) == e) return x;
    return 0;
}
template <int P, int U>
constexpr int lu_ext_y(int e)
{
    constexpr int S = LidUnit<P, U>::side;
    for (int y = -1; y <= S; ++y)
        for (int x = -1; x <= S; ++x)
            if (lu_ext_index<P, U>(x, y) == e) return y;
    return 0;
}

// most members any member touches (the sparse rule needs <= 6)
template <int P, int U>
constexpr int lu_max_degree()
{
    int best = 0;
    for (int u = 0; u < LidUnit<P, U>::NB; ++u) {
        int n = 0;
        for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx)
                if ((dx || dy) && (lu_byte<P, U>(lu_x<P, U>(u) + dx, lu_y<P, U>(u) + dy) >= 0 ||
                                   lu_is_ext<P, U>(lu_x<P, U>(u) + dx, lu_y<P, U>(u) + dy)))
                    ++n;
        if (n > best) best = n;
    }
    return best;
}

}  // namespace fr
