// Canonical simplex lists and filtration values.
//
// Steps 3-5 of Section 3.1 (arXiv 1908.05944): K^d is the set of facets of
// K^(d+1) together with the simplices of Sigma_ortho^d that pass AC2 at their
// orthocentre. The per-atom pass emitted the latter; here both sources are
// mapped to input indices, each tuple sorted ascending, bucketed by its first
// vertex (counting sort over input indices), sorted and de-duplicated inside
// each bucket. A simplex that arrives only as a facet fails AC2 at its own
// orthocentre: it is "attached".
//
// Filtration value Size (Section 2.3): an unattached simplex's closest witness
// is its orthocentre, so Size = OrthoSize; an attached simplex's closest
// witness lies on a face of its witness region, i.e. it is a witness of a
// coface with the same Size (the argument of Lemmas 1 and 2), so Size is the
// smallest Size of its cofaces one dimension up. Ties pick the coface that
// comes first in lexicographic order. OrthoSize is an exact rational of
// 128-bit integers, converted to FP64 with three roundings (relative error
// below 4 * 2^-53).
#include <math.h>

#include <type_traits>

#include "ac_internal.cuh"
#include "ac_bucket.h"
#include "ac_round.h"

namespace ac {

// ---------------------------------------------------------------------------
// helpers

__device__ __forceinline__ void sort_asc(int4& t, int K) {
    // tiny sorting network on the first K components
    auto cs = [](int& a, int& b) {
        if (a > b) {
            int x = a;
            a = b;
            b = x;
        }
    };
    if (K == 2) {
        cs(t.x, t.y);
    } else if (K == 3) {
        cs(t.x, t.y);
        cs(t.y, t.z);
        cs(t.x, t.y);
    } else {
        cs(t.x, t.y);
        cs(t.z, t.w);
        cs(t.x, t.z);
        cs(t.y, t.w);
        cs(t.y, t.z);
    }
}

__device__ __forceinline__ bool less_rest(const int4& a, const int4& b) {
    if (a.y != b.y) return a.y < b.y;
    if (a.z != b.z) return a.z < b.z;
    return a.w < b.w;
}

__device__ __forceinline__ bool same(const int4& a, const int4& b) {
    return a.x == b.x && a.y == b.y && a.z == b.z && a.w == b.w;
}

// Unused tuple slots hold -1 so comparisons ignore them.
__device__ __forceinline__ int4 facet_of(const int4& t, int K, int drop) {
    // t has K+1 valid ascending entries; return the K-tuple without entry drop
    int v[4] = {t.x, t.y, t.z, t.w};
    int o[4] = {-1, -1, -1, -1};
    int w = 0;
    for (int k = 0; k <= K; k++)
        if (k != drop) o[w++] = v[k];
    return make_int4(o[0], o[1], o[2], o[3]);
}

// Items of one dimension: [0, nA) from a list in sorted positions (a4, or a2 for
// edges), then nB * (K + 1) facets of a canonical list of width K + 1. An item
// is an ascending K-tuple of input indices; its bucket is its first vertex. For
// K <= 3 the unused last component carries the flag (1: the simplex passed AC2
// at its orthocentre, 0: a facet); for K = 4 every item is a list item (flag 1).
struct CanonArgs {
    const int4* a4;
    const int2* a2;
    int64_t nA;
    const int4* cof;
    int64_t nB;
    const int32_t* order;  // sorted position -> input index
    int64_t total;
    int64_t* bucket_cnt;   // count pass: items per bucket
    const int64_t* off;    // scatter pass: bucket offsets
    unsigned long long* cursor;
    int4* T;               // scattered items
};

template <int K>
__device__ __forceinline__ int4 canon_item(const CanonArgs& a, int64_t j) {
    int4 t;
    if (j < a.nA) {
        if (K == 2) {
            const int2 e = a.a2[j];
            t = make_int4(a.order[e.x], a.order[e.y], -1, -1);
        } else {
            const int4 e = a.a4[j];
            t = make_int4(a.order[e.x], a.order[e.y], a.order[e.z], K == 4 ? a.order[e.w] : -1);
        }
        sort_asc(t, K);
        if (K < 4) t.w = 1;
    } else {
        const int64_t r = j - a.nA;
        const int64_t row = r / (K + 1);
        const int drop = (int)(r - row * (K + 1));
        t = facet_of(a.cof[row], K, drop);
        t.w = 0;  // K < 4 here: facets exist for K = 2, 3
    }
    return t;
}

// Items in a warp that share a bucket add to its counter once.
template <int K>
__global__ void k_canon_count(CanonArgs a) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = j < a.total;
    const int lane = threadIdx.x & 31;
    const int x = valid ? canon_item<K>(a, j).x : -1 - lane;
    const unsigned peers = __match_any_sync(0xffffffffu, x);
    if (valid && (peers & ((1u << lane) - 1u)) == 0)
        atomicAdd((unsigned long long*)&a.bucket_cnt[x], (unsigned long long)__popc(peers));
}

template <int K>
__global__ void k_canon_scatter(CanonArgs a) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = j < a.total;
    const int lane = threadIdx.x & 31;
    int4 t = make_int4(-1 - lane, 0, 0, 0);
    if (valid) t = canon_item<K>(a, j);
    const unsigned peers = __match_any_sync(0xffffffffu, t.x);
    const int leader = __ffs(peers) - 1;
    unsigned long long base = 0;
    if (valid && lane == leader) base = atomicAdd(&a.cursor[t.x], (unsigned long long)__popc(peers));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (valid) a.T[a.off[t.x] + (int64_t)base + __popc(peers & ((1u << lane) - 1u))] = t;
}

// In-bucket sort and de-duplication, one warp per bucket of up to CSORT_MAX
// items. The rest of each tuple becomes a sort key: K = 2: (y << 1) | flag;
// K = 3: (y << 33) | (z << 1) | flag (y, z < 2^31); K = 4: hi = (y << 32) | z,
// lo = w (flag 1). Keys sit in registers, R = ceil(k/32) per lane (padded to a
// power of two with the largest key), and a bitonic network sorts them:
// exchanges across lanes by shuffles, across a lane's registers directly.
// Equal tuples (the flag bit aside) are then adjacent; the first of each run
// takes the OR of the run's flags and the run is compacted to the front of
// the bucket.
constexpr int CSORT_MAX = 256;
constexpr int CSORT_WARPS = 4;

struct SortSmem {
    unsigned long long ohi[CSORT_MAX];
    unsigned olo[CSORT_MAX];
};

template <int K>
__device__ __forceinline__ void make_key(const int4& t, unsigned long long& hi, unsigned& lo) {
    const unsigned long long y = (unsigned)t.y, z = (unsigned)t.z;
    if (K == 2) {
        hi = (y << 1) | (unsigned)t.w;
        lo = 0u;
    } else if (K == 3) {
        hi = (y << 33) | (z << 1) | (unsigned)t.w;
        lo = 0u;
    } else {
        hi = (y << 32) | z;
        lo = (unsigned)t.w;
    }
}

template <int K, class H>
__device__ __forceinline__ bool key_less(H ah, unsigned al, H bh, unsigned bl) {
    return K == 4 ? (ah < bh || (ah == bh && al < bl)) : ah < bh;
}

// register type of the high key: edges' keys (y << 1 | flag, y < 2^31) fit 32 bits
template <int K>
using KeyHi = typename std::conditional<K == 2, unsigned, unsigned long long>::type;

template <int K, int R>
__device__ __forceinline__ void bitonic_place(SortSmem& S, const int4* __restrict__ T, int64_t a, int k, int lane) {
    using H = KeyHi<K>;
    H h[R];
    unsigned l[R];
#pragma unroll
    for (int r = 0; r < R; r++) {
        const int e = 32 * r + lane;
        if (e < k) {
            unsigned long long hi;
            make_key<K>(T[a + e], hi, l[r]);
            h[r] = (H)hi;
        } else {
            h[r] = (H)~0ull;
            l[r] = ~0u;
        }
    }
    constexpr int N = 32 * R;
#pragma unroll
    for (int size = 2; size <= N; size <<= 1) {
#pragma unroll
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            if (stride >= 32) {
                const int rs = stride >> 5;
#pragma unroll
                for (int r = 0; r < R; r++) {
                    if ((r & rs) == 0) {
                        const int r2 = r | rs;
                        const bool asc = ((32 * r + lane) & size) == 0;
                        if (key_less<K>(h[r2], l[r2], h[r], l[r]) == asc) {
                            const H th = h[r];
                            h[r] = h[r2];
                            h[r2] = th;
                            const unsigned tl = l[r];
                            l[r] = l[r2];
                            l[r2] = tl;
                        }
                    }
                }
            } else {
#pragma unroll
                for (int r = 0; r < R; r++) {
                    const H oh = __shfl_xor_sync(0xffffffffu, h[r], stride);
                    const unsigned ol = K == 4 ? __shfl_xor_sync(0xffffffffu, l[r], stride) : 0u;
                    const bool asc = ((32 * r + lane) & size) == 0;
                    const bool lower = (lane & stride) == 0;
                    // the lower position keeps the smaller key when ascending
                    const bool take = (lower == asc) ? key_less<K>(oh, ol, h[r], l[r]) : key_less<K>(h[r], l[r], oh, ol);
                    if (take) {
                        h[r] = oh;
                        l[r] = ol;
                    }
                }
            }
        }
    }
#pragma unroll
    for (int r = 0; r < R; r++) {
        const int e = 32 * r + lane;
        if (e < k) {
            S.ohi[e] = (unsigned long long)h[r];
            if (K == 4) S.olo[e] = l[r];
        }
    }
}

// Buckets above CSORT_MAX items (rare): one lane, heap sort in place (O(k log k)) then de-duplication.
template <int K>
__device__ void sort_big_bucket(int4* __restrict__ T, int64_t a, int64_t b, int64_t* __restrict__ uniq_g) {
    *uniq_g = sort_unique_bucket<K>(T, a, b);
}

template <int K>
__global__ void __launch_bounds__(CSORT_WARPS * 32) k_canon_sort(int4* __restrict__ T, const int64_t* __restrict__ off,
                                                                  int64_t n, int64_t* __restrict__ uniq, bool unique) {
    __shared__ SortSmem sm[CSORT_WARPS];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    SortSmem& S = sm[w];
    const int64_t warps = (int64_t)gridDim.x * CSORT_WARPS;
    for (int64_t g = (int64_t)blockIdx.x * CSORT_WARPS + w; g < n; g += warps) {
        const int64_t a = off[g];
        const int64_t kb = off[g + 1] - a;
        const int k = kb > CSORT_MAX ? CSORT_MAX + 1 : (int)kb;
        if (unique && k <= 32) {
            // distinct items (nothing to merge), one per lane: each takes its rank among the others
            int4 t = make_int4(0, 0, 0, 0);
            unsigned long long hi = ~0ull;
            unsigned lo = ~0u;
            if (lane < k) {
                t = T[a + lane];
                make_key<K>(t, hi, lo);
            }
            int r = 0;
            for (int u = 0; u < k; u++) {
                const unsigned long long hu = __shfl_sync(0xffffffffu, hi, u);
                const unsigned lu = __shfl_sync(0xffffffffu, lo, u);
                r += key_less<K, unsigned long long>(hu, lu, hi, lo) ? 1 : 0;
            }
            __syncwarp();
            if (lane < k) T[a + r] = t;
            if (lane == 0) uniq[g] = k;
            __syncwarp();
            continue;
        }
        if (k > CSORT_MAX) {
            if (lane == 0) sort_big_bucket<K>(T, a, a + kb, &uniq[g]);
            __syncwarp();
            continue;
        }
        if (k <= 1) {
            if (lane == 0) uniq[g] = k;
            continue;
        }
        if (k <= 32) bitonic_place<K, 1>(S, T, a, k, lane);
        else if (k <= 64) bitonic_place<K, 2>(S, T, a, k, lane);
        else if (k <= 128) bitonic_place<K, 4>(S, T, a, k, lane);
        else bitonic_place<K, 8>(S, T, a, k, lane);
        __syncwarp();
        // same tuple: equal keys without the flag bit (K <= 3), or equal (hi, lo)
        auto same_at = [&](int x, int y) {
            return K == 4 ? (S.ohi[x] == S.ohi[y] && S.olo[x] == S.olo[y]) : (S.ohi[x] >> 1) == (S.ohi[y] >> 1);
        };
        int base = 0;
        for (int i0 = 0; i0 < k; i0 += 32) {
            const int i = i0 + lane;
            bool first = false;
            int fl = 0;
            if (i < k) {
                first = i == 0 || !same_at(i, i - 1);
                if (first) {
                    fl = K == 4 ? 1 : (int)(S.ohi[i] & 1ull);
                    for (int j = i + 1; j < k && same_at(j, i); j++) fl |= (int)(S.ohi[j] & 1ull);
                }
            }
            const unsigned bal = __ballot_sync(0xffffffffu, first);
            if (first) {
                const int pos = base + __popc(bal & ((1u << lane) - 1u));
                const unsigned long long hi = S.ohi[i];
                int4 t;
                t.x = (int)g;
                if (K == 2) {
                    t.y = (int)(hi >> 1);
                    t.z = -1;
                    t.w = fl;
                } else if (K == 3) {
                    t.y = (int)(hi >> 33);
                    t.z = (int)((hi >> 1) & 0xffffffffull);
                    t.w = fl;
                } else {
                    t.y = (int)(hi >> 32);
                    t.z = (int)(unsigned)hi;
                    t.w = (int)S.olo[i];
                }
                T[a + pos] = t;
            }
            base += __popc(bal);
        }
        if (lane == 0) uniq[g] = base;
        __syncwarp();
    }
}

// Slot-parallel output: slot j of bucket g = T[j].x holds unique row j - off[g]
// of the bucket when that is below uniq(g) = uoff[g+1] - uoff[g].
struct CanonWriteArgs {
    const int4* T;
    int64_t total;
    const int64_t* off;
    const int64_t* uoff;
    const int32_t* mol_of;   // input index -> molecule
    const int64_t* mol_off;  // molecule -> first input index
    int4* G;                 // canonical rows, global input indices
    int32_t* out;            // packed rows, per-molecule local indices
    uint8_t* attached;
};

template <int K>
__global__ void k_canon_write(CanonWriteArgs a) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= a.total) return;
    int4 t = a.T[j];
    const int g = t.x;
    const int64_t kk = j - a.off[g];
    const int64_t u0 = a.uoff[g];
    if (kk >= a.uoff[g + 1] - u0) return;
    const int64_t row = u0 + kk;
    const int flag = K == 4 ? 1 : t.w;
    if (K < 4) t.w = -1;
    a.G[row] = t;
    const int base = (int)a.mol_off[a.mol_of[g]];
    a.out[row * K + 0] = t.x - base;
    a.out[row * K + 1] = t.y - base;
    if (K >= 3) a.out[row * K + 2] = t.z - base;
    if (K == 4) a.out[row * K + 3] = t.w - base;
    a.attached[row] = flag ? 0 : 1;
}

// ---------------------------------------------------------------------------
// canonicalise one dimension

using Work = CanonWork;

// the items were unique: the de-duplicated total must equal their number
__global__ void k_check_total(const int64_t* __restrict__ total, int64_t want, unsigned* __restrict__ err) {
    if (*total != want) atomicOr(err, DERR_INTERNAL);
}

template <int K>
static int canon_dim_k(ac_ctx* c, const int4* a4, const int2* a2, int64_t nA, const int4* cof, int64_t nB,
                       SimplexList& L, DevBuf& Gout, Work& w, cudaStream_t s, bool unique) {
    const int64_t n = c->n;
    const int64_t total = nA + nB * (K + 1);
    AC_TRY(w.T.reserve((size_t)(total + 1) * sizeof(int4), s));
    AC_TRY(w.cnt.reserve((size_t)(n + 1) * sizeof(int64_t), s));
    AC_TRY(w.cursor.reserve((size_t)(n + 1) * sizeof(int64_t), s));
    AC_TRY(w.uniq.reserve((size_t)(n + 1) * sizeof(int64_t), s));
    AC_TRY(w.big.reserve((size_t)(n + 1), s));
    AC_TRY(L.v0_off.reserve((size_t)(n + 1) * sizeof(int64_t), s));
    int64_t* cnt = w.cnt.as<int64_t>();
    AC_CUDA(cudaMemsetAsync(cnt, 0, (size_t)(n + 1) * sizeof(int64_t), s));
    AC_CUDA(cudaMemsetAsync(w.cursor.p, 0, (size_t)(n + 1) * sizeof(int64_t), s));
    CanonArgs ca{a4, a2, nA, cof, nB, c->order.as<int32_t>(), total, cnt, cnt, w.cursor.as<unsigned long long>(),
                 w.T.as<int4>()};
    const unsigned gi = (unsigned)((total + 255) / 256);
    if (total > 0) {
        k_canon_count<K><<<gi, 256, 0, s>>>(ca);
        AC_LAUNCHED();
    }
    AC_TRY(scan_exclusive_i64(c, cnt, cnt, n, s));  // bucket offsets, in place
    int64_t* uniq = w.uniq.as<int64_t>();
    if (total > 0) {
        k_canon_scatter<K><<<gi, 256, 0, s>>>(ca);
        AC_LAUNCHED();
    }
    if (n > 0) {
        int dev = 0, sms = 0, per_sm = 0;
        AC_CUDA(cudaGetDevice(&dev));
        AC_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        AC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_canon_sort<K>, CSORT_WARPS * 32, 0));
        // one resident wave, buckets taken grid-stride
        int64_t blocks = (n + CSORT_WARPS - 1) / CSORT_WARPS;
        if (blocks > (int64_t)sms * (per_sm > 0 ? per_sm : 1)) blocks = (int64_t)sms * (per_sm > 0 ? per_sm : 1);
        k_canon_sort<K><<<(unsigned)blocks, CSORT_WARPS * 32, 0, s>>>(w.T.as<int4>(), cnt, n, uniq, unique);
        AC_LAUNCHED();
    }
    int64_t* uoff = L.v0_off.as<int64_t>();
    if (unique)  // every item is a row: the rows start where the buckets do
        AC_CUDA(cudaMemcpyAsync(uoff, cnt, (size_t)(n + 1) * sizeof(int64_t), cudaMemcpyDeviceToDevice, s));
    else
        AC_TRY(scan_exclusive_i64(c, uniq, uoff, n, s));
    int64_t count = L.count;  // a replay keeps the recorded build's count and checks it
    if (c->replaying) {
        AC_TRY(expect_i64(c, uoff + n, count, s));
    } else if (unique) {
        // items emitted once each (by their owner): their number is the count, checked on the device
        count = total;
        k_check_total<<<1, 1, 0, s>>>(uoff + n, total, &c->counters.as<DevCounters>()->err);
        AC_LAUNCHED();
    } else {
        AC_CUDA(cudaMemcpyAsync(c->h_stage, uoff + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        AC_TRY(sync_host(c, s));
        count = c->h_stage[0];
    }
    L.count = count;
    const size_t rows = (size_t)(count > 0 ? count : 1);
    AC_TRY(L.tuples.reserve(rows * K * sizeof(int32_t), s));
    AC_TRY(L.attached.reserve(rows, s));
    AC_TRY(L.f.reserve(rows * sizeof(double), s));
    AC_TRY(L.orthosize.reserve(rows * sizeof(double), s));
    AC_TRY(L.src_dim.reserve(rows, s));
    AC_TRY(L.src_idx.reserve(rows * sizeof(int64_t), s));
    AC_TRY(Gout.reserve(rows * sizeof(int4), s));
    if (total > 0) {
        CanonWriteArgs wa{w.T.as<int4>(), total, cnt, uoff, c->mol_of.as<int32_t>(), c->d_moloff.as<int64_t>(),
                          Gout.as<int4>(), L.tuples.as<int32_t>(), L.attached.as<uint8_t>()};
        k_canon_write<K><<<gi, 256, 0, s>>>(wa);
        AC_LAUNCHED();
    }
    return AC_OK;
}

static int canon_dim(ac_ctx* c, int d, const int4* a4, const int2* a2, int64_t nA, const int4* cof, int64_t nB,
                     SimplexList& L, DevBuf& Gout, Work& w, cudaStream_t s, bool unique = false) {
    switch (d) {
        case 1: return canon_dim_k<2>(c, a4, a2, nA, cof, nB, L, Gout, w, s, unique);
        case 2: return canon_dim_k<3>(c, a4, a2, nA, cof, nB, L, Gout, w, s, unique);
        default: return canon_dim_k<4>(c, a4, a2, nA, cof, nB, L, Gout, w, s, unique);
    }
}

// ---------------------------------------------------------------------------
// K^1 by marks (Step 4 for edges). An edge of K^1 joins two atoms whose grown
// balls meet (its OrthoSize is at most alpha), so its second vertex is an
// entry of the neighbour row of its first vertex (smallest input index); the
// rows list grid-sorted positions in ascending order. The free edges and the
// three edges of every K^2 triangle set bits over those rows (bit OR: a
// duplicate changes nothing, so nothing is sorted or removed), a second mask
// keeps the free edges, and each atom writes its marked entries as rows in
// ascending input order.

struct EdgeMarkArgs {
    const int2* free_e;  // free edges (sorted positions), nA of them
    int64_t nA;
    const int4* tri;     // K^2 rows (global input indices), nB of them
    int64_t nB;
    const int32_t* order;  // sorted position -> input index
    const int32_t* rank;   // input index -> sorted position
    const int64_t* nb_off; // offsets (stride 0) or counts (stride > 0)
    const int32_t* nb;
    int stride;
    int words;             // mask words per atom
    unsigned* m_in;        // per sorted position: entry of the row is an edge of K^1
    unsigned* m_free;      // ... and a free edge
    unsigned long long* rows;  // per input index: distinct marked edges (the atom's row count)
    unsigned* err;
};

__device__ __forceinline__ void edge_row(const EdgeMarkArgs& a, int s, int64_t& off, int& m) {
    if (a.stride) {
        off = (int64_t)s * a.stride;
        m = min((int)a.nb_off[s], a.stride);
    } else {
        off = a.nb_off[s];
        m = (int)(a.nb_off[s + 1] - off);
    }
}

// position of sorted position x in the ascending row [off, off + m), or -1
__device__ __forceinline__ int row_find(const int32_t* __restrict__ nb, int64_t off, int m, int x) {
    int lo = 0, hi = m;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (nb[off + mid] < x) lo = mid + 1;
        else hi = mid;
    }
    return lo < m && nb[off + lo] == x ? lo : -1;
}

// bit e of sorted position su's row mask; the first setting of a bit counts a
// row for input index gu (duplicates leave the count as it is)
__device__ __forceinline__ void mark_bit(const EdgeMarkArgs& a, int su, int gu, int e, bool fr) {
    if (e < 0) {
        atomicOr(a.err, DERR_INTERNAL);  // an edge of K^1 between atoms whose balls do not meet: impossible
        return;
    }
    const int64_t w = (int64_t)su * a.words + (e >> 5);
    const unsigned bit = 1u << (e & 31);
    if (!(atomicOr(&a.m_in[w], bit) & bit)) atomicAdd(&a.rows[gu], 1ull);
    if (fr) atomicOr(&a.m_free[w], bit);
}

// threads [0, nA): one free edge each; then one K^2 triangle (a < b < c) each:
// (a, b) and (a, c) in a's row, (b, c) in b's row
__global__ void k_edge_mark(EdgeMarkArgs a) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= a.nA + a.nB) return;
    int64_t off;
    int m;
    if (j < a.nA) {
        const int2 e = a.free_e[j];
        int gu = a.order[e.x], gv = a.order[e.y];
        int su = e.x, sv = e.y;
        if (gu > gv) {
            su = e.y;
            sv = e.x;
            gu = gv;
        }
        edge_row(a, su, off, m);
        mark_bit(a, su, gu, row_find(a.nb, off, m, sv), true);
        return;
    }
    const int4 t = a.tri[j - a.nA];
    const int sa = a.rank[t.x], sb = a.rank[t.y], sc = a.rank[t.z];
    edge_row(a, sa, off, m);
    const int eb = row_find(a.nb, off, m, sb), ec = row_find(a.nb, off, m, sc);
    int64_t offb;
    int mb;
    edge_row(a, sb, offb, mb);
    const int ebc = row_find(a.nb, offb, mb, sc);
    mark_bit(a, sa, t.x, eb, false);
    mark_bit(a, sa, t.x, ec, false);
    mark_bit(a, sb, t.y, ebc, false);
}

// the marked entries of g's row, ranked by input index: one warp per atom;
// the marked entries' input indices are compacted into shared memory, then
// each marked lane counts the smaller ones
constexpr int EW_WARPS = 4;

__global__ void __launch_bounds__(EW_WARPS * 32) k_edge_write(EdgeMarkArgs a, int64_t n, const int64_t* __restrict__ uoff,
                                                              const int32_t* __restrict__ mol_of,
                                                              const int64_t* __restrict__ mol_off, int4* __restrict__ G,
                                                              int32_t* __restrict__ out, uint8_t* __restrict__ attached,
                                                              uint8_t* __restrict__ endpoint) {
    __shared__ int hs_all[EW_WARPS][MAX_DEGREE];  // an atom's marked entries: at most its row length
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    int* hs = hs_all[wib];
    const int64_t g = (int64_t)blockIdx.x * EW_WARPS + wib;
    if (g >= n) return;
    const int s = a.rank[g];
    const unsigned* mw = a.m_in + (int64_t)s * a.words;
    const unsigned* fw = a.m_free + (int64_t)s * a.words;
    int64_t off;
    int m;
    edge_row(a, s, off, m);
    const int64_t row0 = uoff[g];
    const int base = (int)mol_off[mol_of[g]];
    // pass 1: compact the marked entries (input index, free bit) in entry order
    int c = 0;
    for (int w = 0; w < a.words; w++) {
        const unsigned bits = mw[w];  // the same word for the whole warp
        if (!bits) continue;
        const bool mine = (bits >> lane) & 1u;
        if (mine) {
            const int h = a.order[a.nb[off + 32 * w + lane]];
            hs[c + __popc(bits & ((1u << lane) - 1u))] = h;
        }
        c += __popc(bits);
    }
    __syncwarp();
    // the vertices of K^1 (Step 5: endpoints are in K^0); only ones are written
    if (lane == 0 && c > 0) endpoint[g] = 1;
    // pass 2: rank each compacted entry among the others
    for (int k = lane; k < c; k += 32) {
        const int h = hs[k];
        int r = 0;
        for (int q = 0; q < c; q++) r += hs[q] < h;
        // the free bit of the k-th marked entry
        int rem = k, w = 0;
        unsigned bits = mw[0];
        while (rem >= __popc(bits)) {
            rem -= __popc(bits);
            bits = mw[++w];
        }
        for (int t = 0; t < rem; t++) bits &= bits - 1;
        const int e = __ffs(bits) - 1;
        const int64_t row = row0 + r;
        G[row] = make_int4((int)g, h, -1, -1);
        out[row * 2 + 0] = (int)g - base;
        out[row * 2 + 1] = h - base;
        attached[row] = (fw[w] >> e) & 1u ? 0 : 1;
        endpoint[h] = 1;
    }
}

static int canon_edges_by_marks(ac_ctx* c, cudaStream_t s) {
    const DevCounters& h = c->hc;
    const int64_t n = c->n;
    SimplexList& L = c->K[1];
    Work& w = c->cw;
    const int words = (h.max_degree + 31) / 32 > 0 ? (h.max_degree + 31) / 32 : 1;
    const size_t nn = (size_t)(n > 0 ? n : 1);
    DevBuf& masks = c->scratch[2];
    AC_TRY(masks.reserve(2 * nn * words * sizeof(unsigned), s));
    AC_TRY(w.cnt.reserve((nn + 1) * sizeof(int64_t), s));
    AC_TRY(L.v0_off.reserve((nn + 1) * sizeof(int64_t), s));
    AC_CUDA(cudaMemsetAsync(masks.p, 0, 2 * nn * words * sizeof(unsigned), s));
    int64_t* cnt = w.cnt.as<int64_t>();
    AC_CUDA(cudaMemsetAsync(cnt, 0, nn * sizeof(int64_t), s));
    EdgeMarkArgs a{c->edge_pass.as<int2>(), (int64_t)h.n_edge_pass, c->Gbuf[2].as<int4>(), c->K[2].count,
                   c->order.as<int32_t>(), c->rank.as<int32_t>(), c->nb_cnt.as<int64_t>(), c->nb.as<int32_t>(),
                   c->nb_stride, words, masks.as<unsigned>(), masks.as<unsigned>() + nn * words,
                   reinterpret_cast<unsigned long long*>(cnt), &c->counters.as<DevCounters>()->err};
    const int64_t items = a.nA + a.nB;
    if (items > 0) {
        k_edge_mark<<<(unsigned)((items + 255) / 256), 256, 0, s>>>(a);
        AC_LAUNCHED();
    }
    int64_t* uoff = L.v0_off.as<int64_t>();
    AC_TRY(scan_exclusive_i64(c, cnt, uoff, n, s));
    int64_t count = L.count;
    if (c->replaying) {
        AC_TRY(expect_i64(c, uoff + n, count, s));
    } else {
        AC_CUDA(cudaMemcpyAsync(c->h_stage, uoff + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        AC_TRY(sync_host(c, s));
        count = c->h_stage[0];
    }
    L.count = count;
    const size_t rows = (size_t)(count > 0 ? count : 1);
    AC_TRY(L.tuples.reserve(rows * 2 * sizeof(int32_t), s));
    AC_TRY(L.attached.reserve(rows, s));
    AC_TRY(L.f.reserve(rows * sizeof(double), s));
    AC_TRY(L.orthosize.reserve(rows * sizeof(double), s));
    AC_TRY(L.src_dim.reserve(rows, s));
    AC_TRY(L.src_idx.reserve(rows * sizeof(int64_t), s));
    AC_TRY(c->Gbuf[1].reserve(rows * sizeof(int4), s));
    AC_TRY(w.big.reserve(nn, s));  // endpoint flags of K^1, for K^0
    AC_CUDA(cudaMemsetAsync(w.big.p, 0, nn, s));
    if (n > 0) {
        k_edge_write<<<(unsigned)((n + EW_WARPS - 1) / EW_WARPS), EW_WARPS * 32, 0, s>>>(a, n, uoff, c->mol_of.as<int32_t>(),
                                                                  c->d_moloff.as<int64_t>(), c->Gbuf[1].as<int4>(),
                                                                  L.tuples.as<int32_t>(), L.attached.as<uint8_t>(),
                                                                  w.big.as<uint8_t>());
        AC_LAUNCHED();
    }
    return AC_OK;
}

// ---------------------------------------------------------------------------
// K^2 by marks (Step 3 for triangles), as for edges one dimension up: a
// triangle of K^2 has pairwise-meeting vertices, so its second and third
// vertices are entries p < q of the neighbour row of its first vertex. Each
// atom has a pair mask over its row (bit q (q - 1) / 2 + p), sized by its own
// row length m (m (m - 1) / 2 bits); the free triangles and the four facets of
// every tetrahedron of K^3 set bits, a second mask keeps the free ones, and
// each atom writes its marked pairs in lexicographic input order.

struct TriMarkArgs {
    const int4* free_t;  // free triangles (sorted positions in x, y, z), nA of them
    int64_t nA;
    const int4* tet;     // K^3 rows (global input indices), nB of them
    int64_t nB;
    const int32_t* order;
    const int32_t* rank;
    const int64_t* nb_off;
    const int32_t* nb;
    int stride;
    const int64_t* moff;  // first mask word of each sorted position (n + 1)
    unsigned* m_in;
    unsigned* m_free;
    unsigned long long* rows;  // per input index: distinct marked pairs (the atom's row count)
    unsigned* err;
};

__device__ __forceinline__ void nb_row_of(const int64_t* __restrict__ nb_off, int stride, int s, int64_t& off, int& m) {
    if (stride) {
        off = (int64_t)s * stride;
        m = min((int)nb_off[s], stride);
    } else {
        off = nb_off[s];
        m = (int)(nb_off[s + 1] - off);
    }
}


// The pair-mask layout of the K^2 marks (first word of each sorted position,
// n + 1, into c->pair_moff) from the words per atom the neighbour pass wrote;
// the caller reads the total (pair_moff[n]) with its other sizes.
int plan_pair_masks(ac_ctx* c, const int64_t* pw, cudaStream_t s) {
    const int64_t n = c->n;
    const size_t nn = (size_t)(n > 0 ? n : 1);
    AC_TRY(c->pair_moff.reserve((nn + 1) * sizeof(int64_t), s));
    return scan_exclusive_i64(c, pw, c->pair_moff.as<int64_t>(), n, s);
}

__device__ __forceinline__ void mark_pair(const TriMarkArgs& a, int sa, int ga, int e1, int e2, bool fr) {
    if (e1 < 0 || e2 < 0) {
        atomicOr(a.err, DERR_INTERNAL);  // a triangle of K^2 whose vertices' balls do not meet: impossible
        return;
    }
    const int p = min(e1, e2), q = max(e1, e2);
    const int64_t bit = (int64_t)q * (q - 1) / 2 + p;
    const int64_t w = a.moff[sa] + (bit >> 5);
    const unsigned b = 1u << (bit & 31);
    if (!(atomicOr(&a.m_in[w], b) & b)) atomicAdd(&a.rows[ga], 1ull);
    if (fr) atomicOr(&a.m_free[w], b);
}

// threads [0, nA): one free triangle each; then one K^3 tetrahedron (a < b < c < d)
// each: (a,b,c), (a,b,d), (a,c,d) in a's row, (b,c,d) in b's row
__global__ void k_tri_mark(TriMarkArgs a) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= a.nA + a.nB) return;
    int64_t off;
    int m;
    if (j < a.nA) {
        const int4 t = a.free_t[j];
        int sv[3] = {t.x, t.y, t.z};
        int gv[3] = {a.order[t.x], a.order[t.y], a.order[t.z]};
        int f = 0;  // the vertex with the smallest input index
        if (gv[1] < gv[f]) f = 1;
        if (gv[2] < gv[f]) f = 2;
        const int sa = sv[f], s1 = sv[f == 0 ? 1 : 0], s2 = sv[f == 2 ? 1 : 2];
        nb_row_of(a.nb_off, a.stride, sa, off, m);
        mark_pair(a, sa, gv[f], row_find(a.nb, off, m, s1), row_find(a.nb, off, m, s2), true);
        return;
    }
    const int4 t = a.tet[j - a.nA];
    const int sa = a.rank[t.x], sb = a.rank[t.y], sc = a.rank[t.z], sd = a.rank[t.w];
    nb_row_of(a.nb_off, a.stride, sa, off, m);
    const int pb = row_find(a.nb, off, m, sb), pc = row_find(a.nb, off, m, sc), pd = row_find(a.nb, off, m, sd);
    mark_pair(a, sa, t.x, pb, pc, false);
    mark_pair(a, sa, t.x, pb, pd, false);
    mark_pair(a, sa, t.x, pc, pd, false);
    nb_row_of(a.nb_off, a.stride, sb, off, m);
    mark_pair(a, sb, t.y, row_find(a.nb, off, m, sc), row_find(a.nb, off, m, sd), false);
}

constexpr int TW_WARPS = 4;
constexpr int TW_CAP = 256;  // marked pairs ranked in shared memory; more take the slow path

// The pair (p, q), p < q, of pair-mask bit q (q - 1) / 2 + p. Rows hold at most
// MAX_DEGREE entries, so bit < 2^19: 32-bit arithmetic throughout (a 64-bit
// integer conversion would run on the narrow FP64 pipe).
static_assert((int64_t)MAX_DEGREE * (MAX_DEGREE - 1) / 2 < (1 << 24), "pair bits exact in FP32");
__device__ __forceinline__ void pair_of(int bit, int& p, int& q) {
    int x = (int)((1.0f + sqrtf(1.0f + 8.0f * (float)bit)) * 0.5f);
    while (x * (x - 1) / 2 > bit) x--;
    while ((x + 1) * x / 2 <= bit) x++;
    q = x;
    p = bit - q * (q - 1) / 2;
}

__global__ void __launch_bounds__(TW_WARPS * 32) k_tri_write(TriMarkArgs a, int64_t n, const int64_t* __restrict__ uoff,
                                                             const int32_t* __restrict__ mol_of,
                                                             const int64_t* __restrict__ mol_off, int4* __restrict__ G,
                                                             int32_t* __restrict__ out, uint8_t* __restrict__ attached) {
    __shared__ unsigned long long key_all[TW_WARPS][TW_CAP];
    __shared__ uint8_t fr_all[TW_WARPS][TW_CAP];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int64_t g = (int64_t)blockIdx.x * TW_WARPS + wib;
    if (g >= n) return;
    unsigned long long* key = key_all[wib];
    uint8_t* frs = fr_all[wib];
    const int s = a.rank[g];
    int64_t off;
    int m;
    nb_row_of(a.nb_off, a.stride, s, off, m);
    const int64_t w0 = a.moff[s], w1 = a.moff[s + 1];
    const int64_t row0 = uoff[g];
    const int64_t total = uoff[g + 1] - row0;
    const int base = (int)mol_off[mol_of[g]];
    auto key_of = [&](int64_t bit) {
        int p, q;
        pair_of((int)bit, p, q);
        const unsigned hb = (unsigned)a.order[a.nb[off + p]], hc = (unsigned)a.order[a.nb[off + q]];
        return hb < hc ? ((unsigned long long)hb << 32) | hc : ((unsigned long long)hc << 32) | hb;
    };
    auto emit = [&](unsigned long long k, int64_t r, bool fr) {
        const int y = (int)(k >> 32), z = (int)(k & 0xffffffffu);
        const int64_t row = row0 + r;
        G[row] = make_int4((int)g, y, z, -1);
        out[row * 3 + 0] = (int)g - base;
        out[row * 3 + 1] = y - base;
        out[row * 3 + 2] = z - base;
        attached[row] = fr ? 0 : 1;
    };
    if (total <= TW_CAP) {
        // compact the marked pairs in bit order, then rank them
        int c = 0;
        for (int64_t wb = w0; wb < w1; wb += 32) {
            const int64_t w = wb + lane;
            const unsigned bits = w < w1 ? a.m_in[w] : 0u;
            const int k = __popc(bits);
            int incl = k;
            for (int d = 1; d < 32; d <<= 1) {
                const int v = __shfl_up_sync(0xffffffffu, incl, d);
                if (lane >= d) incl += v;
            }
            int slot = c + incl - k;
            const unsigned frw = bits ? a.m_free[w] : 0u;
            for (unsigned b = bits; b; b &= b - 1) {
                const int t = __ffs(b) - 1;
                key[slot] = key_of((w - w0) * 32 + t);
                frs[slot] = (uint8_t)((frw >> t) & 1u);
                slot++;
            }
            c += __shfl_sync(0xffffffffu, incl, 31);
        }
        __syncwarp();
        for (int k = lane; k < c; k += 32) {
            const unsigned long long kk = key[k];
            int r = 0;
            for (int q = 0; q < c; q++) r += key[q] < kk;
            emit(kk, r, frs[k] != 0);
        }
    } else {
        // many pairs (a very wide row): rank each against all, from the masks
        for (int64_t w = w0; w < w1; w++) {
            const unsigned bits = a.m_in[w];
            const unsigned frw = a.m_free[w];
            for (int t = lane; t < 32; t += 32) {
                if (!((bits >> t) & 1u)) continue;
                const unsigned long long kk = key_of((w - w0) * 32 + t);
                int64_t r = 0;
                for (int64_t w2 = w0; w2 < w1; w2++)
                    for (unsigned b2 = a.m_in[w2]; b2; b2 &= b2 - 1)
                        r += key_of((w2 - w0) * 32 + __ffs(b2) - 1) < kk;
                emit(kk, r, (frw >> t) & 1u);
            }
        }
    }
}

static int canon_tris_by_marks(ac_ctx* c, cudaStream_t s) {
    const DevCounters& h = c->hc;
    const int64_t n = c->n;
    SimplexList& L = c->K[2];
    Work& w = c->cw;
    const size_t nn = (size_t)(n > 0 ? n : 1);
    DevBuf& masks = c->scratch[2];
    AC_TRY(w.cnt.reserve((nn + 1) * sizeof(int64_t), s));
    AC_TRY(L.v0_off.reserve((nn + 1) * sizeof(int64_t), s));
    // first mask word of each sorted position and their total: from the neighbour pass
    const int64_t* moff = c->pair_moff.as<int64_t>();
    int64_t* cnt = w.cnt.as<int64_t>();
    const int64_t words = c->pair_words;
    const size_t mw = (size_t)(words > 0 ? words : 1);
    AC_TRY(masks.reserve(2 * mw * sizeof(unsigned), s));
    AC_CUDA(cudaMemsetAsync(masks.p, 0, 2 * mw * sizeof(unsigned), s));
    AC_CUDA(cudaMemsetAsync(cnt, 0, nn * sizeof(int64_t), s));
    TriMarkArgs a{c->tri_pass.as<int4>(), (int64_t)h.n_tri_pass, c->Gbuf[3].as<int4>(), c->K[3].count,
                  c->order.as<int32_t>(), c->rank.as<int32_t>(), c->nb_cnt.as<int64_t>(), c->nb.as<int32_t>(),
                  c->nb_stride, moff, masks.as<unsigned>(), masks.as<unsigned>() + mw,
                  reinterpret_cast<unsigned long long*>(cnt), &c->counters.as<DevCounters>()->err};
    const int64_t items = a.nA + a.nB;
    if (items > 0) {
        k_tri_mark<<<(unsigned)((items + 255) / 256), 256, 0, s>>>(a);
        AC_LAUNCHED();
    }
    const unsigned wb = (unsigned)((n + TW_WARPS - 1) / TW_WARPS);
    int64_t* uoff = L.v0_off.as<int64_t>();
    AC_TRY(scan_exclusive_i64(c, cnt, uoff, n, s));
    int64_t count = L.count;
    if (c->replaying) {
        AC_TRY(expect_i64(c, uoff + n, count, s));
    } else {
        AC_CUDA(cudaMemcpyAsync(c->h_stage, uoff + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        AC_TRY(sync_host(c, s));
        count = c->h_stage[0];
    }
    L.count = count;
    const size_t rows = (size_t)(count > 0 ? count : 1);
    AC_TRY(L.tuples.reserve(rows * 3 * sizeof(int32_t), s));
    AC_TRY(L.attached.reserve(rows, s));
    AC_TRY(L.f.reserve(rows * sizeof(double), s));
    AC_TRY(L.orthosize.reserve(rows * sizeof(double), s));
    AC_TRY(L.src_dim.reserve(rows, s));
    AC_TRY(L.src_idx.reserve(rows * sizeof(int64_t), s));
    AC_TRY(c->Gbuf[2].reserve(rows * sizeof(int4), s));
    if (n > 0) {
        k_tri_write<<<wb, TW_WARPS * 32, 0, s>>>(a, n, uoff, c->mol_of.as<int32_t>(), c->d_moloff.as<int64_t>(),
                                                 c->Gbuf[2].as<int4>(), L.tuples.as<int32_t>(),
                                                 L.attached.as<uint8_t>());
        AC_LAUNCHED();
    }
    return AC_OK;
}

// Vertices (Step 5): K^0 = endpoints of K^1 (flagged by k_edge_write) + atoms
// whose centre passes AC2.
__global__ void k_vertex_flags(const uint8_t* __restrict__ endpoint, const uint8_t* __restrict__ vert_pass,
                               const int32_t* __restrict__ rank, int64_t n, int64_t* __restrict__ inK) {
    int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= n) return;
    inK[g] = (endpoint[g] || vert_pass[rank[g]]) ? 1 : 0;
}

__global__ void k_vertex_write(const int64_t* __restrict__ voff, const uint8_t* __restrict__ vert_pass,
                               const int32_t* __restrict__ rank, int64_t n, const int32_t* __restrict__ mol_of,
                               const int64_t* __restrict__ mol_off, int4* __restrict__ G, int32_t* __restrict__ out,
                               uint8_t* __restrict__ attached) {
    int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= n) return;
    if (voff[g + 1] == voff[g]) return;
    int64_t r = voff[g];
    G[r] = make_int4((int)g, -1, -1, -1);
    out[r] = (int)(g - mol_off[mol_of[g]]);
    attached[r] = vert_pass[rank[g]] ? 0 : 1;
}

// First row of every molecule in each list: rows of molecule m start at
// v0_off[mol_off[m]]. Lists 0..3 are K^0..K^3, lists 4..6 Sigma^1..Sigma^3.
struct MolRowsArgs {
    const int64_t* v0_off[7];
    const int64_t* mol_off;
    int64_t n_mol;
    int64_t* out;  // 7 x (n_mol + 1)
};

__global__ void k_mol_rows(MolRowsArgs a) {
    const int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (m > a.n_mol) return;
    const int64_t at = a.mol_off[m];
    for (int l = 0; l < 7; l++) a.out[l * (a.n_mol + 1) + m] = a.v0_off[l] ? a.v0_off[l][at] : 0;
}

static int fork_orthosize(ac_ctx* c, int d, cudaStream_t s);

int canonicalise(ac_ctx* c, cudaStream_t s) {
    const DevCounters& h = c->hc;  // counters read at the end of the per-atom pass
    if (h.err & (DERR_OVF_TET | DERR_OVF_TRI | DERR_OVF_EDGE | DERR_OVF_CAND))
        return fail(AC_ERR_CAPACITY, "per-atom output overflow");
    Work& w = c->cw;
    const int64_t n = c->n;
    // K^3
    AC_TRY(canon_dim(c, 3, c->tet_out.as<int4>(), nullptr, (int64_t)h.n_tet_out, nullptr, 0, c->K[3], c->Gbuf[3], w, s,
                     true));
    AC_TRY(fork_orthosize(c, 3, s));
    AC_TRY(stage_mark(c, 4, s));
    // K^2 = unattached triangles + facets of K^3
    AC_TRY(canon_tris_by_marks(c, s));
    AC_TRY(fork_orthosize(c, 2, s));
    AC_TRY(stage_mark(c, 5, s));
    // K^1 = unattached edges + edges of K^2, by marks over the neighbour rows
    AC_TRY(canon_edges_by_marks(c, s));
    AC_TRY(fork_orthosize(c, 1, s));
    // K^0
    {
        SimplexList& L = c->K[0];
        size_t nn = (size_t)(n > 0 ? n : 1);
        AC_TRY(w.big.reserve(nn, s));
        AC_TRY(w.cnt.reserve((nn + 1) * sizeof(int64_t), s));
        AC_TRY(L.v0_off.reserve((nn + 1) * sizeof(int64_t), s));
        uint8_t* endpoint = w.big.as<uint8_t>();  // set by k_edge_write
        int64_t* inK = w.cnt.as<int64_t>();
        if (n > 0) {
            k_vertex_flags<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(endpoint, c->vert_pass.as<uint8_t>(),
                                                                       c->rank.as<int32_t>(), n, inK);
            AC_LAUNCHED();
        }
        int64_t* voff = L.v0_off.as<int64_t>();
        AC_TRY(scan_exclusive_i64(c, inK, voff, n, s));
        int64_t count = L.count;
        if (c->replaying) {
            AC_TRY(expect_i64(c, voff + n, count, s));
        } else {
            AC_CUDA(cudaMemcpyAsync(c->h_stage, voff + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
            AC_TRY(sync_host(c, s));
            count = c->h_stage[0];
        }
        L.count = count;
        size_t rows = (size_t)(count > 0 ? count : 1);
        AC_TRY(L.tuples.reserve(rows * sizeof(int32_t), s));
        AC_TRY(L.attached.reserve(rows, s));
        AC_TRY(L.f.reserve(rows * sizeof(double), s));
        AC_TRY(L.orthosize.reserve(rows * sizeof(double), s));
        AC_TRY(L.src_dim.reserve(rows, s));
        AC_TRY(L.src_idx.reserve(rows * sizeof(int64_t), s));
        AC_TRY(c->Gbuf[0].reserve(rows * sizeof(int4), s));
        if (n > 0) {
            k_vertex_write<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(voff, c->vert_pass.as<uint8_t>(),
                                                                       c->rank.as<int32_t>(), n, c->mol_of.as<int32_t>(),
                                                                       c->d_moloff.as<int64_t>(), c->Gbuf[0].as<int4>(),
                                                                       L.tuples.as<int32_t>(), L.attached.as<uint8_t>());
            AC_LAUNCHED();
        }
    }
    AC_TRY(fork_orthosize(c, 0, s));
    // estimation-pass lists, when kept (single molecule)
    if (c->pc.keep_candidates) {
        for (int d = 1; d <= 3; d++) {
            int64_t m = (int64_t)h.n_cand_out[d];
            // each candidate is emitted once, by its owner
            AC_TRY(canon_dim(c, d, d >= 2 ? c->cand[d].as<int4>() : nullptr, d == 1 ? c->cand[1].as<int2>() : nullptr, m,
                             nullptr, 0, c->C[d], c->CGbuf[d], w, s, true));
        }
    }
    // per-molecule row ranges, copied to the host with the build's last transfer
    MolRowsArgs ma{};
    for (int d = 0; d < 4; d++) ma.v0_off[d] = c->K[d].v0_off.as<int64_t>();
    for (int d = 1; d <= 3; d++) ma.v0_off[3 + d] = c->pc.keep_candidates ? c->C[d].v0_off.as<int64_t>() : nullptr;
    ma.mol_off = c->d_moloff.as<int64_t>();
    ma.n_mol = c->n_mol;
    AC_TRY(w.cursor.reserve((size_t)7 * (c->n_mol + 1) * sizeof(int64_t), s));
    ma.out = w.cursor.as<int64_t>();
    k_mol_rows<<<(unsigned)((c->n_mol + 1 + 127) / 128), 128, 0, s>>>(ma);
    AC_LAUNCHED();
    AC_CUDA(cudaMemcpyAsync(c->h_molrows, ma.out, (size_t)7 * (c->n_mol + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost,
                            s));
    return AC_OK;
}

// Unpack the per-molecule row ranges once the stream has reached the end of the build.
void finish_mol_rows(ac_ctx* c) {
    const size_t m1 = (size_t)c->n_mol + 1;
    for (int d = 0; d < 4; d++) c->K[d].mol_off.assign(c->h_molrows + d * m1, c->h_molrows + (d + 1) * m1);
    if (c->pc.keep_candidates)
        for (int d = 1; d <= 3; d++)
            c->C[d].mol_off.assign(c->h_molrows + (3 + d) * m1, c->h_molrows + (4 + d) * m1);
}

// ---------------------------------------------------------------------------
// OrthoSize (exact) and Size

// OrthoSize of a simplex of global input indices (ascending, K entries) as an
// exact rational num / den in quanta^2 (den > 0).
__device__ void orthosize_rational(const int4* __restrict__ P, const int4& t, int K, i128& num, i128& den);

// OrthoSize in A^2 of a simplex of global input indices (ascending, K entries):
// the numerator (scaled by 2^-20, quanta^2 -> A^2) and the denominator each
// rounded to the nearest double in integer arithmetic, then one FP64 division.
__device__ double orthosize_exact(const int4* __restrict__ P, const int4& t, int K) {
    i128 num, den;
    orthosize_rational(P, t, K, num, den);
    if (K == 1) return i128_to_double_rn(num, -20);  // exact
    return i128_to_double_rn(num, -20) / i128_to_double_rn(den, 0);
}

__device__ void orthosize_rational(const int4* __restrict__ P, const int4& t, int K, i128& num, i128& den) {
    const int4 p0 = P[t.x];
    const long long W0 = p0.w;
    if (K == 1) {
        num = -(i128)W0;
        den = 1;
        return;
    }
    int v[4] = {t.x, t.y, t.z, t.w};
    long long q[3][3], a[3];
    for (int k = 1; k < K; k++) {
        int4 pk = P[v[k]];
        q[k - 1][0] = pk.x - p0.x;
        q[k - 1][1] = pk.y - p0.y;
        q[k - 1][2] = pk.z - p0.z;
        a[k - 1] = q[k - 1][0] * q[k - 1][0] + q[k - 1][1] * q[k - 1][1] + q[k - 1][2] * q[k - 1][2] - pk.w + W0;
    }
    if (K == 2) {
        long long D = q[0][0] * q[0][0] + q[0][1] * q[0][1] + q[0][2] * q[0][2];
        num = (i128)a[0] * a[0] - (i128)4 * D * W0;
        den = (i128)4 * D;
    } else if (K == 3) {
        long long g11 = q[0][0] * q[0][0] + q[0][1] * q[0][1] + q[0][2] * q[0][2];
        long long g22 = q[1][0] * q[1][0] + q[1][1] * q[1][1] + q[1][2] * q[1][2];
        long long g12 = q[0][0] * q[1][0] + q[0][1] * q[1][1] + q[0][2] * q[1][2];
        long long detG = g11 * g22 - g12 * g12;
        long long n1 = g22 * a[0] - g12 * a[1], n2 = g11 * a[1] - g12 * a[0];
        num = (i128)n1 * a[0] + (i128)n2 * a[1] - (i128)4 * detG * W0;
        den = (i128)4 * detG;
    } else {
        long long C[3][3];
        // C_k = q_{k+1} x q_{k+2}
        for (int k = 0; k < 3; k++) {
            const long long* b = q[(k + 1) % 3];
            const long long* d = q[(k + 2) % 3];
            C[k][0] = b[1] * d[2] - b[2] * d[1];
            C[k][1] = b[2] * d[0] - b[0] * d[2];
            C[k][2] = b[0] * d[1] - b[1] * d[0];
        }
        long long D = q[0][0] * C[0][0] + q[0][1] * C[0][1] + q[0][2] * C[0][2];
        long long N[3];
        for (int c = 0; c < 3; c++) N[c] = a[0] * C[0][c] + a[1] * C[1][c] + a[2] * C[2][c];
        i128 nn = (i128)N[0] * N[0] + (i128)N[1] * N[1] + (i128)N[2] * N[2];
        i128 DD = (i128)D * D;
        num = nn - DD * (4 * W0);
        den = DD * 4;
    }
}

__global__ void k_orthosize(const int4* __restrict__ P, const int4* __restrict__ G, int64_t m, int K,
                            const uint8_t* __restrict__ attached, double* __restrict__ os, double* __restrict__ f,
                            int8_t* __restrict__ src_dim, int64_t* __restrict__ src_idx,
                            unsigned long long* __restrict__ fkey) {
    int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= m) return;
    double v = orthosize_exact(P, G[j], K);
    os[j] = v;
    src_dim[j] = (int8_t)(K - 1);
    src_idx[j] = j;
    f[j] = v;
    if (fkey) fkey[j] = attached[j] ? ~0ull : 0ull;
}

__device__ __forceinline__ unsigned long long order_key(double x) {
    unsigned long long b = (unsigned long long)__double_as_longlong(x);
    return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}

__device__ __forceinline__ double key_value(unsigned long long k) {
    unsigned long long b = (k >> 63) ? (k & 0x7fffffffffffffffull) : ~k;
    return __longlong_as_double((long long)b);
}

// row index of tuple t (global indices, K entries) in the canonical list L, or -1
__device__ __forceinline__ int64_t find_row(const int4* __restrict__ L, const int64_t* __restrict__ v0_off, const int4& t) {
    int64_t lo = v0_off[t.x], hi = v0_off[t.x + 1];
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        int4 r = L[mid];
        if (same(r, t)) return mid;
        if (less_rest(r, t)) lo = mid + 1;
        else hi = mid;
    }
    return -1;
}

// pass 1: smallest coface value of every attached face; the row of each
// (coface, facet) that is an attached face is kept for pass 2 (-1 otherwise)
__global__ void k_coface_min(const int4* __restrict__ Cof, const double* __restrict__ fc, int64_t mc, int Kc,
                             const int4* __restrict__ L, const int64_t* __restrict__ v0_off,
                             const uint8_t* __restrict__ attached, unsigned long long* __restrict__ fkey,
                             int64_t* __restrict__ rows) {
    int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= mc) return;
    int4 t = Cof[j];
    unsigned long long key = order_key(fc[j]);
    for (int drop = 0; drop < Kc; drop++) {
        int4 face = facet_of(t, Kc - 1, drop);
        int64_t r = find_row(L, v0_off, face);
        const bool hit = r >= 0 && attached[r];
        rows[j * Kc + drop] = hit ? r : -1;
        if (hit) atomicMin(&fkey[r], key);
    }
}

// pass 2: among cofaces attaining the minimum, the first in lexicographic order
__global__ void k_coface_arg(const double* __restrict__ fc, int64_t mc, int Kc, const int64_t* __restrict__ rows,
                             const unsigned long long* __restrict__ fkey, unsigned long long* __restrict__ arg) {
    int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= mc) return;
    unsigned long long key = order_key(fc[j]);
    for (int drop = 0; drop < Kc; drop++) {
        const int64_t r = rows[j * Kc + drop];
        if (r >= 0 && fkey[r] == key) atomicMin(&arg[r], (unsigned long long)j);
    }
}

__global__ void k_coface_apply(int64_t m, const uint8_t* __restrict__ attached, const unsigned long long* __restrict__ fkey,
                               const unsigned long long* __restrict__ arg, const int8_t* __restrict__ csrc_dim,
                               const int64_t* __restrict__ csrc_idx, double* __restrict__ f, int8_t* __restrict__ src_dim,
                               int64_t* __restrict__ src_idx, unsigned* __restrict__ err) {
    int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= m || !attached[j]) return;
    unsigned long long a = arg[j];
    if (a == ~0ull) {
        // an attached simplex with no coface in the complex cannot occur
        atomicOr(err, DERR_INTERNAL);
        f[j] = __longlong_as_double(0x7ff8000000000000ll);
        return;
    }
    f[j] = key_value(fkey[j]);
    src_dim[j] = csrc_dim[a];
    src_idx[j] = csrc_idx[a];
}

// Sub-complex at alpha2 <= alpha (the filtration restricted): a simplex is in
// K_alpha2 iff Size <= alpha2 (Section 2.4). Size is the OrthoSize of the
// simplex's source (itself when unattached, else the coface its value came
// from), compared exactly: num <= A2 den.
__global__ void k_subcomplex(const int4* __restrict__ P, const int4* __restrict__ const* G, const int8_t* __restrict__ src_dim,
                             const int64_t* __restrict__ src_idx, int64_t first, int64_t m, long long A2,
                             uint8_t* __restrict__ flags, unsigned long long* __restrict__ n_in) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    bool in = false;
    if (j < m) {
        const int sd = src_dim[first + j];
        const int4 t = G[sd][src_idx[first + j]];
        i128 num, den;
        orthosize_rational(P, t, sd + 1, num, den);
        in = num <= (i128)A2 * den;
        flags[j] = in ? 1 : 0;
    }
    const unsigned b = __ballot_sync(0xffffffffu, in);
    if ((threadIdx.x & 31) == 0 && b) atomicAdd(n_in, (unsigned long long)__popc(b));
}

int subcomplex_flags(ac_ctx* c, int dim, int64_t first, int64_t m, double alpha2, uint8_t* flags, int64_t* count,
                     cudaStream_t s) {
    const long long A2 = (long long)nearbyint(alpha2 * 1048576.0);
    AC_TRY(c->scratch[6].reserve(sizeof(unsigned long long) + 4 * sizeof(int4*), s));
    unsigned long long* n_in = c->scratch[6].as<unsigned long long>();
    const int4** g = reinterpret_cast<const int4**>(n_in + 1);
    const int4* gh[4];
    for (int d = 0; d < 4; d++) gh[d] = c->Gbuf[d].as<int4>();
    AC_CUDA(cudaMemcpyAsync(g, gh, sizeof(gh), cudaMemcpyHostToDevice, s));
    AC_CUDA(cudaMemsetAsync(n_in, 0, sizeof(unsigned long long), s));
    if (m > 0) {
        SimplexList& L = c->K[dim];
        k_subcomplex<<<(unsigned)((m + 255) / 256), 256, 0, s>>>(c->P.as<int4>(), g, L.src_dim.as<int8_t>(),
                                                                  L.src_idx.as<int64_t>(), first, m, A2, flags, n_in);
        AC_LAUNCHED();
    }
    unsigned long long h = 0;
    AC_CUDA(cudaMemcpyAsync(&h, n_in, sizeof(h), cudaMemcpyDeviceToHost, s));
    AC_CUDA(cudaStreamSynchronize(s));
    *count = (int64_t)h;
    return AC_OK;
}

// opt.host_results: list d (rows, the selected filtration values, attached
// flags) to its page-locked host block, on the context's copy stream (the
// device-to-host link, about 190 GB/s here, is the limit, so the copies start
// as early as they can and never hold up the filtration): the rows and flags
// once the list's rows are written (after stream `from`), the values once
// they are final (after stream `from`); compute_filtration joins the copies.
static int copy_after(ac_ctx* c, cudaStream_t from) {
    AC_CUDA(cudaEventRecord(c->ev_copy, from));
    AC_CUDA(cudaStreamWaitEvent(c->copy, c->ev_copy, 0));
    c->copy_forked = true;
    return AC_OK;
}

static int copy_rows_to_host(ac_ctx* c, int d, cudaStream_t from) {
    if (!c->opt.host_results) return AC_OK;
    const SimplexList& L = c->K[d];
    const int64_t m = L.count;
    const int k = d + 1;
    AC_TRY(host_block_for(c, d, hres_bytes_for(m, k)));
    char* b = static_cast<char*>(c->hres[d]);
    AC_TRY(copy_after(c, from));
    AC_CUDA(cudaMemcpyAsync(b, L.tuples.p, (size_t)m * k * sizeof(int32_t), cudaMemcpyDeviceToHost, c->copy));
    AC_CUDA(cudaMemcpyAsync(b + hres_a_off(m, k), L.attached.p, (size_t)m, cudaMemcpyDeviceToHost, c->copy));
    return AC_OK;
}

static int copy_values_to_host(ac_ctx* c, int d, cudaStream_t from) {
    if (!c->opt.host_results) return AC_OK;
    const SimplexList& L = c->K[d];
    const int64_t m = L.count;
    const int k = d + 1;
    char* b = static_cast<char*>(c->hres[d]);
    const DevBuf& f = c->opt.filtration == AC_FILTRATION_ORTHOSIZE ? L.orthosize : L.f;
    AC_TRY(copy_after(c, from));
    AC_CUDA(cudaMemcpyAsync(b + hres_f_off(m, k), f.p, (size_t)m * sizeof(double), cudaMemcpyDeviceToHost, c->copy));
    return AC_OK;
}

// The filtration of list d on the side stream, as soon as the list's rows are
// final, overlapping the canonicalisation of the lower dimensions: OrthoSize
// (with the initial Size, source and coface key), then for d < 3 the two
// coface passes over K^(d+1), whose values are final by then (the side stream
// ran its passes first). compute_filtration joins the side stream. Each pass
// has its own buffers, reserved here on the build's stream before the fork.
static int fork_orthosize(ac_ctx* c, int d, cudaStream_t s) {
    SimplexList& L = c->K[d];
    const int64_t m = L.count;
    if (m == 0) return AC_OK;
    SimplexList* U = d < 3 ? &c->K[d + 1] : nullptr;
    const int64_t mu = U ? U->count : 0;
    AC_TRY(c->fkey[d].reserve((size_t)m * sizeof(unsigned long long), s));
    if (U) {
        AC_TRY(c->fargs[d].reserve((size_t)m * sizeof(unsigned long long), s));
        if (mu > 0) AC_TRY(c->frows[d].reserve((size_t)mu * (d + 2) * sizeof(int64_t), s));
    }
    AC_TRY(copy_rows_to_host(c, d, s));
    AC_CUDA(cudaEventRecord(c->ev_fork, s));
    cudaStream_t t = c->side;
    AC_CUDA(cudaStreamWaitEvent(t, c->ev_fork, 0));
    unsigned long long* keyb = c->fkey[d].as<unsigned long long>();
    k_orthosize<<<(unsigned)((m + 127) / 128), 128, 0, t>>>(c->P.as<int4>(), c->Gbuf[d].as<int4>(), m, d + 1,
                                                            L.attached.as<uint8_t>(), L.orthosize.as<double>(),
                                                            L.f.as<double>(), L.src_dim.as<int8_t>(),
                                                            L.src_idx.as<int64_t>(), keyb);
    AC_LAUNCHED();
    c->os_forked = true;
    if (!U) return copy_values_to_host(c, d, t);
    unsigned long long* argb = c->fargs[d].as<unsigned long long>();
    AC_CUDA(cudaMemsetAsync(argb, 0xff, (size_t)m * sizeof(unsigned long long), t));
    if (mu > 0) {
        const unsigned nbk = (unsigned)((mu + 127) / 128);
        int64_t* rows = c->frows[d].as<int64_t>();
        k_coface_min<<<nbk, 128, 0, t>>>(c->Gbuf[d + 1].as<int4>(), U->f.as<double>(), mu, d + 2, c->Gbuf[d].as<int4>(),
                                         L.v0_off.as<int64_t>(), L.attached.as<uint8_t>(), keyb, rows);
        AC_LAUNCHED();
        k_coface_arg<<<nbk, 128, 0, t>>>(U->f.as<double>(), mu, d + 2, rows, keyb, argb);
        AC_LAUNCHED();
    }
    k_coface_apply<<<(unsigned)((m + 127) / 128), 128, 0, t>>>(
        m, L.attached.as<uint8_t>(), keyb, argb, U->src_dim.as<int8_t>(), U->src_idx.as<int64_t>(), L.f.as<double>(),
        L.src_dim.as<int8_t>(), L.src_idx.as<int64_t>(), &c->counters.as<DevCounters>()->err);
    AC_LAUNCHED();
    return copy_values_to_host(c, d, t);
}

// Size of every list (Section 2.3): computed on the side stream as the lists
// were finished (fork_orthosize); the build's stream waits for it here.
int compute_filtration(ac_ctx* c, cudaStream_t s) {
    if (c->os_forked) {
        AC_CUDA(cudaEventRecord(c->ev_join, c->side));
        AC_CUDA(cudaStreamWaitEvent(s, c->ev_join, 0));
        c->os_forked = false;
    }
    if (c->copy_forked) {
        AC_CUDA(cudaEventRecord(c->ev_cjoin, c->copy));
        AC_CUDA(cudaStreamWaitEvent(s, c->ev_cjoin, 0));
        c->copy_forked = false;
    }
    return AC_OK;
}

}  // namespace ac
