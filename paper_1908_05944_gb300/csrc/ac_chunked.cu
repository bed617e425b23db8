// Out-of-core build (Section 4.6, "handling large data sizes"): the molecule
// is cut into slabs along z; each slab, with a halo of the atoms within reach
// of it, is one ordinary device build; each build keeps the simplices whose
// first (smallest input index) vertex lies in its slab, and those shares are
// placed in host memory in first-vertex order.
//
// Why a slab's share is exact: for a simplex sigma with first vertex v, every
// coface of sigma contains v, so all of their vertices, and every atom that
// can violate AC2 at one of their orthocentres (a common neighbour of their
// vertices, Section 4.4), have grown balls that meet v's: |Z - Z_v| <= 2h in
// quanta. The halo holds all of them, the subset keeps the global input order
// (so index-based symbolic perturbation breaks ties the same way), and every
// decision is exact, so sigma's membership, attached flag and Size come out
// as in the build of the whole molecule.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <functional>
#include <memory>
#include <new>
#include <thread>
#include <vector>

#include "ac_internal.cuh"

namespace {

template <class T>
struct HostArr {
    std::unique_ptr<T[]> p;
    int64_t n = 0;
    bool reset(int64_t count) {
        p.reset(count > 0 ? new (std::nothrow) T[(size_t)count] : nullptr);
        n = count;
        return count == 0 || p != nullptr;
    }
};

double now_ms() {
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

}  // namespace

struct ac_chunked {
    HostArr<int32_t> t[4];
    HostArr<double> f[4];
    HostArr<uint8_t> a[4];
    int64_t count[4] = {0, 0, 0, 0};
    ac_chunked_stats st{};
};

namespace ac {
namespace {

int host_threads() { return (int)std::max(1u, std::min(16u, std::thread::hardware_concurrency())); }

// fn(t, begin, end) over T contiguous ranges of [0, n), one thread each
void parallel_ranges(int64_t n, int T, const std::function<void(int, int64_t, int64_t)>& fn) {
    if (T <= 1 || n < 65536) {
        fn(0, 0, n);
        for (int t = 1; t < T; t++) fn(t, n, n);
        return;
    }
    std::vector<std::thread> pool;
    for (int t = 0; t < T; t++) pool.emplace_back(fn, t, n * t / T, n * (t + 1) / T);
    for (auto& th : pool) th.join();
}

struct SlabPlan {
    std::vector<int64_t> thr;  // slab k: thr[k] <= Z < thr[k + 1]
    int64_t reach = 0;         // 2 h in quanta
    std::vector<int32_t> Z;    // quantised z of every atom
    int64_t zmin = 0, zmax = -1;
};

// Quantised z and the largest weight of every atom, with the same input
// checks as the device quantisation (so a chunked build fails where ac_create
// would); the reach 2h follows.
int quantise_z(const double* centres, const double* radii, int64_t n, double alpha, SlabPlan& P) {
    if (n < 0) return fail(AC_ERR_INVALID_ARG, "n < 0");
    if (n >= ((int64_t)1 << 31) - 1) return fail(AC_ERR_INVALID_ARG, "n out of range");
    if (n > 0 && (!centres || !radii)) return fail(AC_ERR_INVALID_ARG, "centres/radii NULL");
    if (!std::isfinite(alpha)) return fail(AC_ERR_INVALID_ARG, "alpha not finite");
    if (std::fabs(alpha) > 16.0) return fail(AC_ERR_RANGE, "|alpha| must be at most 16 A^2");
    P.Z.resize((size_t)n);
    const int T = host_threads();
    struct Part {
        int64_t bad_invalid = -1, bad_range = -1, wmax = 0, zmin = INT64_MAX, zmax = INT64_MIN;
    };
    std::vector<Part> part((size_t)T);
    const double lim = 1048576.0;
    parallel_ranges(n, T, [&](int t, int64_t i0, int64_t i1) {
        Part& q = part[(size_t)t];
        for (int64_t i = i0; i < i1; i++) {
            const double x = centres[3 * i], y = centres[3 * i + 1], z = centres[3 * i + 2], r = radii[i];
            if (!(std::isfinite(x) && std::isfinite(y) && std::isfinite(z) && std::isfinite(r)) || !(r > 0.0)) {
                if (q.bad_invalid < 0) q.bad_invalid = i;
                continue;
            }
            if (std::fabs(x) > lim || std::fabs(y) > lim || std::fabs(z) > lim || r > 64.0) {
                if (q.bad_range < 0) q.bad_range = i;
                continue;
            }
            const int64_t R = (int64_t)std::nearbyint(r * 1024.0);
            const double cq = 1073741823.0;  // |quantised coordinate| < 2^30, as the device build requires
            if (R < 1 || R > 4096 || std::fabs(std::nearbyint(x * 1024.0)) > cq || std::fabs(std::nearbyint(y * 1024.0)) > cq ||
                std::fabs(std::nearbyint(z * 1024.0)) > cq) {
                if (q.bad_range < 0) q.bad_range = i;
                continue;
            }
            q.wmax = std::max(q.wmax, R * R);
            const int64_t Zq = (int64_t)std::nearbyint(z * 1024.0);
            P.Z[(size_t)i] = (int32_t)Zq;
            q.zmin = std::min(q.zmin, Zq);
            q.zmax = std::max(q.zmax, Zq);
        }
    });
    int64_t bad_invalid = -1, bad_range = -1;
    int64_t wmax = 0, zmin = INT64_MAX, zmax = INT64_MIN;
    for (const Part& q : part) {  // ranges in order: the first bad atom of the first range that has one
        if (bad_invalid < 0) bad_invalid = q.bad_invalid;
        if (bad_range < 0) bad_range = q.bad_range;
        wmax = std::max(wmax, q.wmax);
        zmin = std::min(zmin, q.zmin);
        zmax = std::max(zmax, q.zmax);
    }
    char b[160];
    if (bad_invalid >= 0) {
        snprintf(b, sizeof(b), "atom %lld: non-finite value or radius <= 0", (long long)bad_invalid);
        return fail(AC_ERR_INVALID_ARG, b);
    }
    if (bad_range >= 0) {
        snprintf(b, sizeof(b), "atom %lld: |coordinate| >= 2^20 A or radius outside (0, 4] A after quantisation",
                 (long long)bad_range);
        return fail(AC_ERR_RANGE, b);
    }
    const int64_t A = (int64_t)std::nearbyint(alpha * 1048576.0);
    const int64_t H2 = (n > 0 ? wmax : 0) + A;
    if (H2 > ((int64_t)1 << 24)) return fail(AC_ERR_RANGE, "r_max^2 + alpha exceeds 16 A^2");
    int64_t hq = 0;  // ceil(sqrt(H2))
    if (H2 > 0) {
        hq = (int64_t)std::floor(std::sqrt((double)H2));
        while (hq * hq < H2) hq++;
        while (hq > 0 && (hq - 1) * (hq - 1) >= H2) hq--;
    }
    // two grown balls meet only if |dZ| <= sqrt(s_i) + sqrt(s_x) <= 2 sqrt(H2)
    P.reach = 2 * hq;
    P.zmin = n > 0 ? zmin : 0;
    P.zmax = n > 0 ? zmax : -1;
    P.thr.clear();
    return AC_OK;
}

// Histogram of the quantised z of the atoms with lo <= Z < hi: bins of
// 2^shift quanta from lo, at most 2^22 + 1 of them.
struct ZHist {
    int shift = 0;
    int64_t lo = 0, bins = 0;
    std::vector<std::atomic<uint32_t>> h;
};

void z_histogram(const SlabPlan& P, int64_t lo, int64_t hi, ZHist& H) {
    const int64_t span = hi - 1 - lo;
    H.shift = 0;
    while ((span >> H.shift) >= ((int64_t)1 << 22)) H.shift++;
    H.lo = lo;
    H.bins = (span >> H.shift) + 1;
    std::vector<std::atomic<uint32_t>> hist((size_t)H.bins);
    for (auto& x : hist) x.store(0, std::memory_order_relaxed);
    parallel_ranges((int64_t)P.Z.size(), host_threads(), [&](int, int64_t i0, int64_t i1) {
        for (int64_t i = i0; i < i1; i++) {
            const int64_t Z = P.Z[(size_t)i];
            if (Z >= lo && Z < hi) hist[(size_t)((Z - lo) >> H.shift)].fetch_add(1, std::memory_order_relaxed);
        }
    });
    H.h.swap(hist);
}

// Greedy cuts of the atoms with lo <= Z < hi into slabs of at most max_core
// atoms (more only when one bin holds more): P.thr, from the lowest to one past
// the highest z in the range (empty when the range holds no atom).
void cut_slabs(SlabPlan& P, int64_t lo, int64_t hi, int64_t max_core) {
    P.thr.clear();
    lo = std::max(lo, P.zmin);
    hi = std::min(hi, P.zmax + 1);
    if (lo >= hi) return;
    ZHist H;
    z_histogram(P, lo, hi, H);
    int64_t first = -1, last = -1;
    for (int64_t bi = 0; bi < H.bins; bi++)
        if (H.h[(size_t)bi].load(std::memory_order_relaxed)) {
            if (first < 0) first = bi;
            last = bi;
        }
    if (first < 0) return;
    P.thr.push_back(lo);
    int64_t run = 0;
    for (int64_t bi = first; bi <= last; bi++) {
        const int64_t h = H.h[(size_t)bi].load(std::memory_order_relaxed);
        if (h == 0) continue;
        if (run > 0 && run + h > max_core) {
            P.thr.push_back(lo + (bi << H.shift));
            run = 0;
        }
        run += h;
    }
    P.thr.push_back(hi);
}

// n_parts ranges of z holding about n / n_parts atoms each (cuts at bin
// boundaries of the histogram of all atoms: a part may hold more, or none,
// when many atoms share one bin): thr[0] = zmin, thr[n_parts] = zmax + 1.
void cut_parts(const SlabPlan& P, int64_t n_parts, std::vector<int64_t>& thr) {
    const int64_t n = (int64_t)P.Z.size();
    thr.assign((size_t)n_parts + 1, P.zmax + 1);
    thr[0] = P.zmin;
    if (n == 0) return;
    ZHist H;
    z_histogram(P, P.zmin, P.zmax + 1, H);
    int64_t cum = 0, bi = 0;
    for (int64_t k = 1; k < n_parts; k++) {
        const int64_t target = (k * n + n_parts - 1) / n_parts;  // atoms below cut k
        while (bi < H.bins && cum < target) cum += H.h[(size_t)bi++].load(std::memory_order_relaxed);
        thr[(size_t)k] = std::max(thr[(size_t)k - 1], std::min(P.zmin + (bi << H.shift), P.zmax + 1));
    }
}

// The slab cut of a whole molecule.
int plan_slabs(const double* centres, const double* radii, int64_t n, double alpha, int64_t max_core, SlabPlan& P) {
    if (n >= 0 && n < ((int64_t)1 << 31) - 1 && (n == 0 || (centres && radii)) && max_core < 1)
        return fail(AC_ERR_INVALID_ARG, "max_core_atoms < 1");
    AC_TRY(quantise_z(centres, radii, n, alpha, P));
    if (n > 0) cut_slabs(P, P.zmin, P.zmax + 1, max_core);
    return AC_OK;
}

// keep[i] = 1 if row i's first vertex lies in the slab
__global__ void k_slab_keep(const int32_t* __restrict__ tuples, int64_t count, int k, const uint8_t* __restrict__ core,
                            int64_t* __restrict__ keep) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < count) keep[i] = core[tuples[i * k]];
}

// the kept rows, in order, with input indices of the whole molecule
__global__ void k_slab_gather(const int32_t* __restrict__ tuples, const double* __restrict__ f,
                              const uint8_t* __restrict__ att, int64_t count, int k, const uint8_t* __restrict__ core,
                              const int64_t* __restrict__ pos, const int32_t* __restrict__ gidx,
                              int32_t* __restrict__ t_out, double* __restrict__ f_out, uint8_t* __restrict__ a_out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count || !core[tuples[i * k]]) return;
    const int64_t p = pos[i];
    for (int j = 0; j < k; j++) t_out[p * k + j] = gidx[tuples[i * k + j]];
    f_out[p] = f[i];
    a_out[p] = att[i];
}

struct Share {
    HostArr<int32_t> t;
    HostArr<double> f;
    HostArr<uint8_t> a;
};

// Device buffers reused across the slabs (released on the caller's stream).
struct SlabBufs {
    DevBuf gidx, core, keep, pos, t, f, a;
};

void parallel_for(int64_t n, int threads, const std::function<void(int64_t)>& fn) {
    if (threads <= 1 || n <= 1) {
        for (int64_t i = 0; i < n; i++) fn(i);
        return;
    }
    std::atomic<int64_t> next{0};
    std::vector<std::thread> pool;
    const int T = (int)std::min<int64_t>(threads, n);
    for (int t = 0; t < T; t++)
        pool.emplace_back([&] {
            for (int64_t i; (i = next.fetch_add(1)) < n;) fn(i);
        });
    for (auto& th : pool) th.join();
}

// One slab: build the subset, keep its share of every list, copy it to host memory.
int build_slab(const double* centres, const double* radii, const int32_t* members, int64_t m, int64_t lo, int64_t hi,
               const SlabPlan& P, double alpha, const ac_options& opt, cudaStream_t s, double* h_xyz, double* h_r,
               int32_t* h_g, uint8_t* h_core, int64_t* h_cnt, SlabBufs& B, Share* out) {
    parallel_ranges(m, host_threads(), [&](int, int64_t j0, int64_t j1) {
        for (int64_t j = j0; j < j1; j++) {
            const int64_t i = members[j];
            h_xyz[3 * j] = centres[3 * i];
            h_xyz[3 * j + 1] = centres[3 * i + 1];
            h_xyz[3 * j + 2] = centres[3 * i + 2];
            h_r[j] = radii[i];
            h_g[j] = (int32_t)i;
            const int64_t Z = P.Z[(size_t)i];
            h_core[j] = (uint8_t)(Z >= lo && Z < hi);
        }
    });
    ac_ctx* c = nullptr;
    AC_TRY(ac_create(h_xyz, h_r, m, alpha, &opt, &c));
    struct Guard {
        ac_ctx* c;
        ~Guard() { ac_destroy(c); }
    } guard{c};
    int rc;
    if ((rc = B.gidx.reserve((size_t)m * sizeof(int32_t), s)) || (rc = B.core.reserve((size_t)m, s))) return rc;
    AC_CUDA(cudaMemcpyAsync(B.gidx.p, h_g, (size_t)m * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    AC_CUDA(cudaMemcpyAsync(B.core.p, h_core, (size_t)m, cudaMemcpyHostToDevice, s));
    AC_TRY(ac_build(c, s));
    for (int d = 0; d < 4; d++) {
        const int32_t* dt = nullptr;
        const double* df = nullptr;
        const uint8_t* da = nullptr;
        int64_t cnt = 0;
        AC_TRY(ac_get_simplices(c, d, -1, &dt, &cnt));
        AC_TRY(ac_filtration_values(c, d, -1, &df, &cnt));
        AC_TRY(ac_attached_flags(c, d, -1, &da, &cnt));
        Share& S = out[d];
        if (cnt == 0) {
            S.t.reset(0);
            S.f.reset(0);
            S.a.reset(0);
            continue;
        }
        const int k = d + 1;
        if ((rc = B.keep.reserve((size_t)(cnt + 1) * sizeof(int64_t), s)) ||
            (rc = B.pos.reserve((size_t)(cnt + 1) * sizeof(int64_t), s)))
            return rc;
        const unsigned nb = (unsigned)((cnt + 255) / 256);
        k_slab_keep<<<nb, 256, 0, s>>>(dt, cnt, k, B.core.as<uint8_t>(), B.keep.as<int64_t>());
        AC_LAUNCHED();
        AC_TRY(scan_exclusive_i64(c, B.keep.as<int64_t>(), B.pos.as<int64_t>(), cnt, s));
        AC_CUDA(cudaMemcpyAsync(h_cnt, B.pos.as<int64_t>() + cnt, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        AC_CUDA(cudaMemcpyAsync(h_cnt + 1, &c->counters.as<DevCounters>()->err, sizeof(unsigned),
                                cudaMemcpyDeviceToHost, s));
        AC_CUDA(cudaStreamSynchronize(s));
        if (reinterpret_cast<const unsigned*>(h_cnt + 1)[0] & DERR_TIMEOUT)
            return fail(AC_ERR_TIMEOUT, "a bounded device wait (scan look-back) ran out");
        const int64_t kept = h_cnt[0];
        if (!S.t.reset(kept * k) || !S.f.reset(kept) || !S.a.reset(kept))
            return fail(AC_ERR_OOM, "host allocation of a slab's share failed");
        if (kept == 0) continue;
        // first touch of the fresh pages on many threads, not inside the copy
        parallel_ranges(kept, host_threads(), [&](int, int64_t r0, int64_t r1) {
            std::fill(S.t.p.get() + r0 * k, S.t.p.get() + r1 * k, 0);
            std::fill(S.f.p.get() + r0, S.f.p.get() + r1, 0.0);
            std::fill(S.a.p.get() + r0, S.a.p.get() + r1, (uint8_t)0);
        });
        if ((rc = B.t.reserve((size_t)kept * k * sizeof(int32_t), s)) || (rc = B.f.reserve((size_t)kept * 8, s)) ||
            (rc = B.a.reserve((size_t)kept, s)))
            return rc;
        k_slab_gather<<<nb, 256, 0, s>>>(dt, df, da, cnt, k, B.core.as<uint8_t>(), B.pos.as<int64_t>(),
                                         B.gidx.as<int32_t>(), B.t.as<int32_t>(), B.f.as<double>(),
                                         B.a.as<uint8_t>());
        AC_LAUNCHED();
        AC_CUDA(cudaMemcpyAsync(S.t.p.get(), B.t.p, (size_t)kept * k * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        AC_CUDA(cudaMemcpyAsync(S.f.p.get(), B.f.p, (size_t)kept * sizeof(double), cudaMemcpyDeviceToHost, s));
        AC_CUDA(cudaMemcpyAsync(S.a.p.get(), B.a.p, (size_t)kept, cudaMemcpyDeviceToHost, s));
    }
    AC_CUDA(cudaStreamSynchronize(s));
    return AC_OK;
}

}  // namespace
}  // namespace ac

using namespace ac;

extern "C" int ac_chunk_plan(const double* centres, const double* radii, int64_t n, double alpha,
                             int64_t max_core_atoms, int64_t* thresholds, int64_t cap, int64_t* n_chunks,
                             int64_t* reach) {
    if (!n_chunks || !reach || (cap > 0 && !thresholds)) return fail(AC_ERR_INVALID_ARG, "NULL output");
    SlabPlan P;
    AC_TRY(plan_slabs(centres, radii, n, alpha, max_core_atoms, P));
    const int64_t k = P.thr.empty() ? 0 : (int64_t)P.thr.size() - 1;
    *n_chunks = k;
    *reach = P.reach;
    if (cap < k + 1) return fail(AC_ERR_INVALID_ARG, "thresholds array too small (needs n_chunks + 1)");
    std::copy(P.thr.begin(), P.thr.end(), thresholds);
    return AC_OK;
}

namespace ac {
namespace {

// One share of one list: rows (count, k) in first-vertex order, host memory.
struct ShareView {
    const int32_t* t;
    const double* f;
    const uint8_t* a;
    int64_t rows;
};

// Placement: the rows of every first vertex come from one share, contiguous
// and in order; the work is cut into pieces of whole runs of rows with the
// same first vertex, many per share. Fails if two shares (or two runs of one
// share) hold rows of the same first vertex, or a first vertex is outside
// [0, n).
int place(int64_t n, int d, const std::vector<ShareView>& shares, std::vector<int64_t>& off, ac_chunked* R) {
    const int k = d + 1;
    const int threads = host_threads();
    struct Piece {
        int64_t c, r0, r1;
    };
    std::vector<Piece> pieces;
    int64_t rows_in = 0;
    for (int64_t c = 0; c < (int64_t)shares.size(); c++) {
        const ShareView& S = shares[(size_t)c];
        rows_in += S.rows;
        const int64_t rows = S.rows, per = std::max<int64_t>(8192, rows / (4 * threads) + 1);
        for (int64_t r0 = 0; r0 < rows;) {
            int64_t r1 = std::min(rows, r0 + per);
            while (r1 < rows && S.t[(size_t)(r1 * k)] == S.t[(size_t)((r1 - 1) * k)]) r1++;
            pieces.push_back({c, r0, r1});
            r0 = r1;
        }
    }
    off.assign((size_t)n + 1, 0);
    std::atomic<int> bad{0};
    // every share strictly increasing, row after row (lexicographic)
    std::atomic<int> unordered{0};
    parallel_for((int64_t)pieces.size(), threads, [&](int64_t pi) {
        const Piece& q = pieces[(size_t)pi];
        const int32_t* t = shares[(size_t)q.c].t;
        for (int64_t r = std::max<int64_t>(q.r0, 1); r < q.r1; r++) {
            const int32_t* x = t + (r - 1) * k;
            const int32_t* y = t + r * k;
            int j = 0;
            while (j < k && x[j] == y[j]) j++;
            if (j == k || x[j] > y[j]) {
                unordered.store(1);
                return;
            }
        }
    });
    if (unordered.load()) return fail(AC_ERR_INVALID_ARG, "a share's rows are not in lexicographic order");
    auto runs = [&](const Piece& q, const std::function<void(int32_t, int64_t, int64_t)>& fn) {
        const ShareView& S = shares[(size_t)q.c];
        for (int64_t r = q.r0; r < q.r1;) {
            const int32_t v = S.t[(size_t)(r * k)];
            int64_t e = r + 1;
            while (e < q.r1 && S.t[(size_t)(e * k)] == v) e++;
            if (v < 0 || v >= n) bad.store(1);
            else fn(v, r, e);
            r = e;
        }
    };
    parallel_for((int64_t)pieces.size(), threads, [&](int64_t pi) {
        runs(pieces[(size_t)pi], [&](int32_t v, int64_t r, int64_t e) { off[(size_t)v + 1] = e - r; });
    });
    if (bad.load()) return fail(AC_ERR_INVALID_ARG, "a row's first vertex is outside [0, n)");
    {
        // inclusive prefix over off[1..n] in ranges: range sums, their prefix, then each range
        std::vector<int64_t> part((size_t)threads + 1, 0);
        parallel_ranges(n, threads, [&](int t, int64_t v0, int64_t v1) {
            int64_t acc = 0;
            for (int64_t v = v0; v < v1; v++) acc += off[(size_t)v + 1];
            part[(size_t)t + 1] = acc;
        });
        for (int t = 0; t < threads; t++) part[(size_t)t + 1] += part[(size_t)t];
        parallel_ranges(n, threads, [&](int t, int64_t v0, int64_t v1) {
            int64_t acc = part[(size_t)t];
            for (int64_t v = v0; v < v1; v++) {
                acc += off[(size_t)v + 1];
                off[(size_t)v + 1] = acc;
            }
        });
    }
    const int64_t total = n > 0 ? off[(size_t)n] : 0;
    if (total != rows_in)
        return fail(AC_ERR_INVALID_ARG, "two shares hold rows of the same first vertex (or a share is not in order)");
    if (!R->t[d].reset(total * k) || !R->f[d].reset(total) || !R->a[d].reset(total))
        return fail(AC_ERR_OOM, "host allocation of the result failed");
    R->count[d] = total;
    parallel_for((int64_t)pieces.size(), threads, [&](int64_t pi) {
        const ShareView& S = shares[(size_t)pieces[(size_t)pi].c];
        runs(pieces[(size_t)pi], [&](int32_t v, int64_t r, int64_t e) {
            const int64_t p = off[(size_t)v];
            std::copy(S.t + r * k, S.t + e * k, R->t[d].p.get() + p * k);
            std::copy(S.f + r, S.f + e, R->f[d].p.get() + p);
            std::copy(S.a + r, S.a + e, R->a[d].p.get() + p);
        });
    });
    return AC_OK;
}

// The rows whose first vertex has lo <= Z < hi, built in slabs of at most
// max_core atoms of that range (each with its halo, from all n atoms),
// placed in first-vertex order into res (host). P holds Z and the reach.
int build_range(const double* centres, const double* radii, int64_t n, double alpha, const ac_options& o,
                int64_t max_core, SlabPlan& P, int64_t lo, int64_t hi, cudaStream_t s, ac_chunked* res) {
    const double t0 = now_ms();
    cut_slabs(P, lo, hi, max_core);
    const int64_t K = P.thr.empty() ? 0 : (int64_t)P.thr.size() - 1;
    // members of slab k (with halo): thr[k] - reach <= Z < thr[k+1] + reach, in input order;
    // T ranges of atoms counted apart, so each range writes its members in order
    auto range_of = [&](int64_t Z, int64_t& k0, int64_t& k1) {
        // first k with thr[k+1] + reach > Z, last k with thr[k] - reach <= Z
        k0 = std::upper_bound(P.thr.begin() + 1, P.thr.end(), Z - P.reach) - (P.thr.begin() + 1);
        k1 = (std::upper_bound(P.thr.begin(), P.thr.end() - 1, Z + P.reach) - P.thr.begin()) - 1;
    };
    const int T = host_threads();
    std::vector<int64_t> tcnt((size_t)T * (size_t)K, 0), tcore((size_t)T * (size_t)K, 0);
    if (K > 0)
        parallel_ranges(n, T, [&](int t, int64_t i0, int64_t i1) {
            int64_t* cnt = tcnt.data() + (size_t)t * K;
            int64_t* core = tcore.data() + (size_t)t * K;
            for (int64_t i = i0; i < i1; i++) {
                const int64_t Z = P.Z[(size_t)i];
                int64_t k0, k1;
                range_of(Z, k0, k1);
                for (int64_t k = k0; k <= k1; k++) {
                    cnt[k]++;
                    if (Z >= P.thr[(size_t)k] && Z < P.thr[(size_t)k + 1]) core[k]++;
                }
            }
        });
    std::vector<int64_t> moff((size_t)K + 1, 0);
    int64_t core_max = 0, sub_max = 0;
    for (int64_t k = 0; k < K; k++) {
        int64_t m = 0, nc = 0;
        for (int t = 0; t < T; t++) {
            const int64_t c = tcnt[(size_t)t * K + k];
            tcnt[(size_t)t * K + k] = moff[(size_t)k] + m;  // this range's first slot in slab k
            m += c;
            nc += tcore[(size_t)t * K + k];
        }
        moff[(size_t)k + 1] = moff[(size_t)k] + m;
        sub_max = std::max(sub_max, m);
        core_max = std::max(core_max, nc);
    }
    std::vector<int32_t> members((size_t)moff[(size_t)K]);
    if (K > 0)
        parallel_ranges(n, T, [&](int t, int64_t i0, int64_t i1) {
            int64_t* cur = tcnt.data() + (size_t)t * K;
            for (int64_t i = i0; i < i1; i++) {
                int64_t k0, k1;
                range_of(P.Z[(size_t)i], k0, k1);
                for (int64_t k = k0; k <= k1; k++) members[(size_t)cur[k]++] = (int32_t)i;
            }
        });
    const double t1 = now_ms();

    // pinned staging for one slab
    double *h_xyz = nullptr, *h_r = nullptr;
    int32_t* h_g = nullptr;
    uint8_t* h_core = nullptr;
    int64_t* h_cnt = nullptr;
    struct Pinned {
        void* p[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
        ~Pinned() {
            for (void* q : p)
                if (q) cudaFreeHost(q);
        }
    } pin;
    std::vector<std::unique_ptr<Share[]>> shares((size_t)K);
    if (K > 0) {
        const size_t sm = (size_t)std::max<int64_t>(sub_max, 1);
        if (cudaMallocHost(&pin.p[0], sm * 3 * sizeof(double)) != cudaSuccess ||
            cudaMallocHost(&pin.p[1], sm * sizeof(double)) != cudaSuccess ||
            cudaMallocHost(&pin.p[2], sm * sizeof(int32_t)) != cudaSuccess ||
            cudaMallocHost(&pin.p[3], sm) != cudaSuccess || cudaMallocHost(&pin.p[4], 4 * sizeof(int64_t)) != cudaSuccess)
            return cuda_fail(cudaGetLastError(), "cudaMallocHost of the slab staging", __FILE__, __LINE__);
        h_xyz = static_cast<double*>(pin.p[0]);
        h_r = static_cast<double*>(pin.p[1]);
        h_g = static_cast<int32_t*>(pin.p[2]);
        h_core = static_cast<uint8_t*>(pin.p[3]);
        h_cnt = static_cast<int64_t*>(pin.p[4]);
        SlabBufs B;
        for (int64_t k = 0; k < K; k++) {
            shares[(size_t)k].reset(new (std::nothrow) Share[4]);
            if (!shares[(size_t)k]) return fail(AC_ERR_OOM, "host allocation failed");
            const int64_t m = moff[(size_t)k + 1] - moff[(size_t)k];
            AC_TRY(build_slab(centres, radii, members.data() + moff[(size_t)k], m, P.thr[(size_t)k],
                              P.thr[(size_t)k + 1], P, alpha, o, s, h_xyz, h_r, h_g, h_core, h_cnt, B,
                              shares[(size_t)k].get()));
        }
        AC_CUDA(cudaStreamSynchronize(s));
    }
    const double t2 = now_ms();
    std::vector<int64_t> off;
    for (int d = 0; d < 4; d++) {
        std::vector<ShareView> views;
        for (int64_t c = 0; c < K; c++) {
            const Share& S = shares[(size_t)c][d];
            views.push_back({S.t.p.get(), S.f.p.get(), S.a.p.get(), S.f.n});
        }
        AC_TRY(place(n, d, views, off, res));
    }
    const double t3 = now_ms();
    ac_chunked_stats& st = res->st;
    st.n_chunks = K;
    st.reach = P.reach;
    st.core_max = core_max;
    st.subset_max = sub_max;
    st.subset_total = moff[(size_t)K];
    st.ms_plan += t1 - t0;
    st.ms_device = t2 - t1;
    st.ms_assemble = t3 - t2;
    return AC_OK;
}

}  // namespace
}  // namespace ac

extern "C" int ac_build_chunked(const double* centres, const double* radii, int64_t n, double alpha,
                                const ac_options* opt, int64_t max_core_atoms, void* stream, ac_chunked** out) {
    if (!out) return fail(AC_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    ac_options o{};
    if (opt) o = *opt;
    if (o.keep_candidates) return fail(AC_ERR_INVALID_ARG, "keep_candidates is not available in a chunked build");
    cudaStream_t s = (cudaStream_t)stream;
    StreamScope scope(s);
    std::unique_ptr<ac_chunked> res(new (std::nothrow) ac_chunked());
    if (!res) return fail(AC_ERR_OOM, "host allocation failed");
    const double t0 = now_ms();
    SlabPlan P;
    AC_TRY(plan_slabs(centres, radii, n, alpha, max_core_atoms, P));
    res->st.ms_plan = now_ms() - t0;
    AC_TRY(build_range(centres, radii, n, alpha, o, max_core_atoms, P, P.zmin, P.zmax + 1, s, res.get()));
    *out = res.release();
    return AC_OK;
}

extern "C" int ac_part_plan(const double* centres, const double* radii, int64_t n, double alpha, int64_t n_parts,
                            int64_t* thresholds, int64_t* reach) {
    if (!thresholds || !reach) return fail(AC_ERR_INVALID_ARG, "NULL output");
    if (n_parts < 1) return fail(AC_ERR_INVALID_ARG, "n_parts < 1");
    SlabPlan P;
    AC_TRY(quantise_z(centres, radii, n, alpha, P));
    std::vector<int64_t> thr;
    cut_parts(P, n_parts, thr);
    std::copy(thr.begin(), thr.end(), thresholds);
    *reach = P.reach;
    return AC_OK;
}

extern "C" int ac_build_part(const double* centres, const double* radii, int64_t n, double alpha,
                             const ac_options* opt, int64_t n_parts, int64_t part, int64_t max_core_atoms, void* stream,
                             ac_chunked** out) {
    if (!out) return fail(AC_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (n_parts < 1 || part < 0 || part >= n_parts) return fail(AC_ERR_INVALID_ARG, "part outside [0, n_parts)");
    if (max_core_atoms < 1) return fail(AC_ERR_INVALID_ARG, "max_core_atoms < 1");
    ac_options o{};
    if (opt) o = *opt;
    if (o.keep_candidates) return fail(AC_ERR_INVALID_ARG, "keep_candidates is not available in a part build");
    cudaStream_t s = (cudaStream_t)stream;
    StreamScope scope(s);
    std::unique_ptr<ac_chunked> res(new (std::nothrow) ac_chunked());
    if (!res) return fail(AC_ERR_OOM, "host allocation failed");
    const double t0 = now_ms();
    SlabPlan P;
    AC_TRY(quantise_z(centres, radii, n, alpha, P));
    std::vector<int64_t> thr;
    cut_parts(P, n_parts, thr);
    res->st.ms_plan = now_ms() - t0;
    AC_TRY(build_range(centres, radii, n, alpha, o, max_core_atoms, P, thr[(size_t)part], thr[(size_t)part + 1], s,
                       res.get()));
    *out = res.release();
    return AC_OK;
}

extern "C" int ac_merge_parts(int64_t n, int64_t n_parts, const int64_t* counts, const int32_t* const* tuples,
                              const double* const* f, const uint8_t* const* attached, ac_chunked** out) {
    if (!out) return fail(AC_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (n < 0 || n_parts < 0 || (n_parts > 0 && (!counts || !tuples || !f || !attached)))
        return fail(AC_ERR_INVALID_ARG, "bad argument");
    std::unique_ptr<ac_chunked> res(new (std::nothrow) ac_chunked());
    if (!res) return fail(AC_ERR_OOM, "host allocation failed");
    const double t0 = now_ms();
    std::vector<int64_t> off;
    for (int d = 0; d < 4; d++) {
        std::vector<ShareView> views;
        for (int64_t p = 0; p < n_parts; p++) {
            const int64_t c = counts[4 * p + d];
            if (c < 0 || (c > 0 && (!tuples[4 * p + d] || !f[4 * p + d] || !attached[4 * p + d])))
                return fail(AC_ERR_INVALID_ARG, "a share has a negative count or a NULL array");
            views.push_back({tuples[4 * p + d], f[4 * p + d], attached[4 * p + d], c});
        }
        AC_TRY(place(n, d, views, off, res.get()));
    }
    res->st.n_chunks = n_parts;
    res->st.ms_assemble = now_ms() - t0;
    *out = res.release();
    return AC_OK;
}

extern "C" int ac_chunked_simplices(const ac_chunked* res, int dim, const int32_t** tuples, const double** f,
                                    const uint8_t** attached, int64_t* count) {
    if (!res || dim < 0 || dim > 3) return fail(AC_ERR_INVALID_ARG, "bad argument");
    if (tuples) *tuples = res->t[dim].p.get();
    if (f) *f = res->f[dim].p.get();
    if (attached) *attached = res->a[dim].p.get();
    if (count) *count = res->count[dim];
    return AC_OK;
}

extern "C" int ac_chunked_info(const ac_chunked* res, ac_chunked_stats* out) {
    if (!res || !out) return fail(AC_ERR_INVALID_ARG, "NULL argument");
    *out = res->st;
    return AC_OK;
}

extern "C" void ac_chunked_free(ac_chunked* res) { delete res; }
