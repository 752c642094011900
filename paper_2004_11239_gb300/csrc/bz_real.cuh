// Index helpers of the real-data form (BZ_DATA_REAL) shared by its reductions: the Nyquist set S
// (modes with an index N/2, i.e. signed -N/2), the mirror -k (mod N per axis), and the position
// of a mode of S in the [3][N][N] family layout of the Nyquist sums X and table C
// (k1 = -N/2 -> family 0 [k2][k3]; else k3 = -N/2 -> family 2 [k1][k2]; else family 1 [k1][k3]).
#pragma once

#include <cstddef>

namespace bz {

__device__ __forceinline__ bool nyquist(int i1, int i2, int i3, int N) {
    const int h = N / 2;
    return i1 == h || i2 == h || i3 == h;
}
__device__ __forceinline__ size_t mirror(int i1, int i2, int i3, int N) {
    const int m1 = (N - i1) % N, m2 = (N - i2) % N, m3 = (N - i3) % N;
    return ((size_t)m1 * N + m2) * N + m3;
}
__device__ __forceinline__ int family_index(int i1, int i2, int i3, int N) {
    const int h = N / 2;
    if (i1 == h) return i2 * N + i3;
    if (i3 == h) return 2 * N * N + i1 * N + i2;
    return N * N + i1 * N + i3;
}

}  // namespace bz
