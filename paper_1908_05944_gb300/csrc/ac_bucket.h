// In-place sort and de-duplication of one large bucket of canonical tuples
// (all tuples of the bucket share their first vertex x), done by one thread:
// heap sort on (y, z[, w]), O(k log k) steps with no scratch memory, then equal
// tuples merged. Used for the rare buckets above the warp sort's size limit
// (the candidate lists of point clouds with hundreds of neighbours per point
// reach buckets of 10^5 tuples). Host and device: the CPU tests compile it
// with g++ and check it against a plain sort.
#pragma once

#include <stdint.h>

#if defined(__CUDACC__)
#define AC_BUCKET_HD __host__ __device__ __forceinline__
#else
#define AC_BUCKET_HD inline
#endif

namespace ac {

// Order of the tuples in a bucket: y, then z, then (K = 4) w. For K < 4, w
// is a flag, not part of the key.
template <int K, class Tup>
AC_BUCKET_HD bool tuple_less(const Tup& u, const Tup& v) {
    if (u.y != v.y) return u.y < v.y;
    if (u.z != v.z) return u.z < v.z;
    return K == 4 && u.w < v.w;
}

template <int K, class Tup>
AC_BUCKET_HD bool tuple_same(const Tup& u, const Tup& v) {
    return u.y == v.y && u.z == v.z && (K != 4 || u.w == v.w);
}

// Move H[root] down the max-heap H[0 .. n) to its place.
template <int K, class Tup>
AC_BUCKET_HD void heap_sift_down(Tup* H, int64_t root, int64_t n) {
    const Tup v = H[root];
    int64_t i = root;
    for (;;) {
        int64_t c = 2 * i + 1;
        if (c >= n) break;
        if (c + 1 < n && tuple_less<K>(H[c], H[c + 1])) c++;
        if (!tuple_less<K>(v, H[c])) break;
        H[i] = H[c];
        i = c;
    }
    H[i] = v;
}

// Sorts T[a .. b) in increasing order, then compacts each run of equal tuples
// to its first (for K < 4 that one takes the OR of the run's flags in w) at
// the front of the range; returns the number of distinct tuples.
template <int K, class Tup>
AC_BUCKET_HD int64_t sort_unique_bucket(Tup* T, int64_t a, int64_t b) {
    Tup* H = T + a;
    const int64_t n = b - a;
    for (int64_t r = n / 2 - 1; r >= 0; r--) heap_sift_down<K>(H, r, n);
    for (int64_t m = n - 1; m > 0; m--) {
        const Tup top = H[0];
        H[0] = H[m];
        H[m] = top;
        heap_sift_down<K>(H, 0, m);
    }
    int64_t w = 0;
    for (int64_t i = 0; i < n; i++) {
        const Tup v = H[i];
        if (w > 0 && tuple_same<K>(H[w - 1], v)) {
            if (K < 4) H[w - 1].w |= v.w;
        } else {
            H[w++] = v;
        }
    }
    return w;
}

}  // namespace ac
