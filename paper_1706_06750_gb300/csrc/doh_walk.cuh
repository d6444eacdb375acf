// doh_walk.cuh -- the lattice walker of the detector response of Eq. 8
// (used by the response kernel, k_detector.cu).
//
// Second derivatives from two concatenated step-s Scharr operators are
// separable on the lattice {-2s, -s, 0, s, 2s}^2 (integer taps, common
// denominator 1024 s^2 folded into `scale` with the normalisation).  A walker
// owns one column x and DOH_WK consecutive lattice rows y = py + s k,
// k = k0 .. k0 + DOH_WK - 1, of one residue py: it loads each lattice row's
// five taps x - 2s .. x + 2s (reflected into the image) DOH_DPD rows ahead,
// filters it horizontally once, and combines the last five filtered rows.
#pragma once

#include "kaze_internal.h"

namespace kz {

constexpr int DOH_WK = 24;  // outputs per walker (consecutive lattice rows)
constexpr int DOH_DPD = 4;  // lattice rows of loads kept in flight

// ld(ptr) loads one float (the read-only path for a level written by an
// earlier launch); emit(j, v) sees the walker's j-th response.
template <typename Load, typename Emit>
__device__ __forceinline__ void doh_walk(const float* __restrict__ L, float* __restrict__ D, int pitch, int w, int h,
                                         int s, float scale, int x, int py, int k0, Load ld, Emit emit)
{
    int cx[5];
#pragma unroll
    for (int a = 0; a < 5; ++a) cx[a] = reflect_index(x + (a - 2) * s, w);
    // lattice rows k0 - 2 .. k0 + WK + 1 of residue py; element offsets within
    // the level plane fit 32 bits
    constexpr int NM = DOH_WK + 4;
    float buf[DOH_DPD + 1][5];
#pragma unroll
    for (int m = 0; m < DOH_DPD; ++m) {
        const int ro = reflect_index(py + s * (k0 + m - 2), h) * pitch;
#pragma unroll
        for (int a = 0; a < 5; ++a) buf[m][a] = ld(L + (unsigned)(ro + cx[a]));
    }
    float hd[5], hs[5], hx[5];
#pragma unroll
    for (int m = 0; m < NM; ++m) {
        if (m + DOH_DPD < NM) {
            const int ro = reflect_index(py + s * (k0 + m + DOH_DPD - 2), h) * pitch;
#pragma unroll
            for (int a = 0; a < 5; ++a) buf[(m + DOH_DPD) % (DOH_DPD + 1)][a] = ld(L + (unsigned)(ro + cx[a]));
        }
        const float* v = buf[m % (DOH_DPD + 1)];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            hd[q] = hd[q + 1];
            hs[q] = hs[q + 1];
            hx[q] = hx[q + 1];
        }
        doh_lattice_row(v[0], v[1], v[2], v[3], v[4], hd[4], hs[4], hx[4]);
        if (m < 4) continue;
        const int y = py + s * (k0 + m - 4);
        if (y >= h) break;
        const float r = doh_value(hd, hs, hx, scale);
        D[(unsigned)(y * pitch + x)] = r;
        emit(m - 4, r);
    }
}

// Walkers of one level: (segment, residue, column), the column fastest.
__host__ __device__ inline int doh_segments(int h, int s) { return ((h + s - 1) / s + DOH_WK - 1) / DOH_WK; }

}  // namespace kz
