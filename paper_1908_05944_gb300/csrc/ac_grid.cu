// Grid binning and neighbour lists (Section 4.2 of arXiv 1908.05944).
//
// Atoms are binned in a uniform grid of cell side ~ h = sqrt(r_max^2 + alpha)
// and sorted by cell so that every cell is a contiguous run (the grid itself
// is never stored per atom). The sort is a counting sort on the cell key (a
// single-digit radix sort: histogram, exclusive scan, scatter) followed by an
// in-cell ordering by input index, so the sorted order is deterministic.
//
// Neighbours: x is a neighbour of i when the grown balls (squared radius
// W + A) of i and x meet, |P_i - P_x| <= sqrt(W_i + A) + sqrt(W_x + A), decided
// exactly in integers. Every vertex pair of a simplex with OrthoSize <= alpha
// and every ball that can violate AC2 at its orthocentre satisfies this with
// each vertex (the orthocentre lies in every vertex's grown ball and in the
// violator's), so these lists are all the later stages search. Pairs are up
// to 2h apart, hence the stencil reach ceil(2h / cell) cells per axis (not the
// single ring of adjacent cells of Section 4.3).
#include "ac_internal.cuh"

namespace ac {

__global__ void k_cell_keys(const int4* __restrict__ P, const int32_t* __restrict__ mol_of,
                            const MolGrid* __restrict__ grids, int cell, int64_t n, uint32_t* __restrict__ cell_of,
                            uint32_t* __restrict__ cell_cnt) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int4 p = P[i];
    MolGrid g = grids[mol_of[i]];
    int cx = (p.x - g.org[0]) / cell, cy = (p.y - g.org[1]) / cell, cz = (p.z - g.org[2]) / cell;
    uint32_t c = (uint32_t)(g.cell_base + ((int64_t)cz * g.dims[1] + cy) * g.dims[0] + cx);
    cell_of[i] = c;
    atomicAdd(&cell_cnt[c], 1u);
}

__global__ void k_scatter(const uint32_t* __restrict__ cell_of, const uint32_t* __restrict__ cell_start, int64_t n,
                          uint32_t* __restrict__ cursor, int32_t* __restrict__ order) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint32_t c = cell_of[i];
    uint32_t slot = cell_start[c] + atomicAdd(&cursor[c], 1u);
    order[slot] = (int32_t)i;
}

// Order each cell's run by input index (runs are short: a few atoms).
__global__ void k_sort_cells(const uint32_t* __restrict__ cell_start, int64_t n_cells, int32_t* __restrict__ order) {
    int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n_cells) return;
    uint32_t a = cell_start[c], b = cell_start[c + 1];
    for (uint32_t i = a + 1; i < b; i++) {
        int32_t v = order[i];
        uint32_t j = i;
        while (j > a && order[j - 1] > v) {
            order[j] = order[j - 1];
            j--;
        }
        order[j] = v;
    }
}

__global__ void k_gather(const int32_t* __restrict__ order, const int4* __restrict__ P,
                         const int32_t* __restrict__ mol_of, int64_t n, int4* __restrict__ Ps,
                         int32_t* __restrict__ mol_s, int32_t* __restrict__ rank) {
    int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    int32_t i = order[s];
    Ps[s] = P[i];
    mol_s[s] = mol_of[i];
    rank[i] = (int32_t)s;
}

int build_grid(ac_ctx* c, cudaStream_t s) {
    const int64_t n = c->n;
    size_t nn = (size_t)(n > 0 ? n : 1);
    AC_TRY(c->cell_of.reserve(nn * sizeof(uint32_t), s));
    AC_TRY(c->cell_cnt.reserve((size_t)(c->n_cells + 1) * sizeof(uint32_t), s));
    AC_TRY(c->cell_start.reserve((size_t)(c->n_cells + 1) * sizeof(uint32_t), s));
    AC_TRY(c->order.reserve(nn * sizeof(int32_t), s));
    AC_TRY(c->rank.reserve(nn * sizeof(int32_t), s));
    AC_TRY(c->Ps.reserve(nn * sizeof(int4), s));
    AC_TRY(c->mol_s.reserve(nn * sizeof(int32_t), s));
    uint32_t* cnt = c->cell_cnt.as<uint32_t>();
    uint32_t* start = c->cell_start.as<uint32_t>();
    AC_CUDA(cudaMemsetAsync(cnt, 0, (size_t)c->n_cells * sizeof(uint32_t), s));
    if (n == 0) {
        AC_CUDA(cudaMemsetAsync(start, 0, (size_t)(c->n_cells + 1) * sizeof(uint32_t), s));
        return AC_OK;
    }
    const unsigned nb = (unsigned)((n + 255) / 256);
    k_cell_keys<<<nb, 256, 0, s>>>(c->P.as<int4>(), c->mol_of.as<int32_t>(), c->grids.as<MolGrid>(), c->pc.cell, n,
                                   c->cell_of.as<uint32_t>(), cnt);
    AC_LAUNCHED();
    AC_TRY(scan_exclusive_u32_to_u32(c, cnt, start, c->n_cells, s));
    AC_CUDA(cudaMemsetAsync(cnt, 0, (size_t)c->n_cells * sizeof(uint32_t), s));
    k_scatter<<<nb, 256, 0, s>>>(c->cell_of.as<uint32_t>(), start, n, cnt, c->order.as<int32_t>());
    AC_LAUNCHED();
    k_sort_cells<<<(unsigned)((c->n_cells + 255) / 256), 256, 0, s>>>(start, c->n_cells, c->order.as<int32_t>());
    AC_LAUNCHED();
    k_gather<<<nb, 256, 0, s>>>(c->order.as<int32_t>(), c->P.as<int4>(), c->mol_of.as<int32_t>(), n, c->Ps.as<int4>(),
                                c->mol_s.as<int32_t>(), c->rank.as<int32_t>());
    AC_LAUNCHED();
    return AC_OK;
}

// Do the closed grown balls of two atoms meet?  t = D - s_i - s_x; they meet iff
// t <= 0 or t^2 <= 4 s_i s_x (s = W + A >= 0).
__device__ __forceinline__ bool grown_meet(int64_t D, int64_t si, int64_t sx) {
    int64_t t = D - si - sx;
    return t <= 0 || t * t <= 4 * si * sx;
}

// L(i) for every atom (Section 4.2: the atoms of the cells around the atom's
// own), one thread per atom. The thread walks the stencil rows (one z, one y,
// a run of cells along x: a contiguous range of the sorted atoms) in (z, y)
// order, four candidates per step (their int4 loads issued together), so L(i)
// comes out in increasing sorted position. Neighbouring threads hold atoms of
// the same or adjacent cells, so their candidate loads overlap in L1.
// SMALL: the stencil spans less than NB_SPAN_SMALL quanta per axis, and a
// pair's test runs in 32-bit integers: squared distances below 2^32, exact
// 64-bit products of 32-bit factors. Otherwise the test runs in 64-bit
// integers, with the coordinate differences bounded first (very coarse cells).
// MODE: NB_COUNT counts L(i); NB_CSR writes it at the offsets nb_off (a scan of
// the counts); NB_PADDED counts it and writes its first NB_STRIDE entries to the
// row nb[s * NB_STRIDE ..] in the same pass.
enum { NB_COUNT = 0, NB_CSR = 1, NB_PADDED = 2 };
constexpr int NB_UNROLL = 4;
constexpr int NB_THREADS = 256;
constexpr int NB_SPAN_SMALL = 37837;  // 3 * 37837^2 < 2^32

struct GridView {
    const int4* Ps;
    const int32_t* mol_s;
    const MolGrid* grids;
    const uint32_t* cell_start;
};

// Does candidate o meet the atom p (grown squared radius si)? Sets the
// coincidence error for a second atom at p's centre.
template <bool SMALL>
__device__ __forceinline__ bool nb_meet(const int4& p, int64_t si, int32_t si32, int A32, const PredConst& pc,
                                        const int4& o, DevCounters* cnt) {
    if (SMALL) {
        // |differences| < NB_SPAN_SMALL: the squared distance fits 32 bits
        const int dx = o.x - p.x, dy = o.y - p.y, dz = o.z - p.z;
        const uint32_t D = (uint32_t)(dx * dx) + (uint32_t)(dy * dy) + (uint32_t)(dz * dz);
        const int sx = o.w + A32;
        if (D == 0) {
            atomicOr(&cnt->err, DERR_COINCIDENT);
            return false;
        }
        if (sx < 0) return false;
        // meet iff D <= si + sx or (D - si - sx)^2 <= 4 si sx
        const uint32_t ss = (uint32_t)(si32 + sx), e = D - ss;
        return D <= ss || (uint64_t)e * e <= (uint64_t)(4u * (uint32_t)si32) * (uint32_t)sx;
    } else {
        const int64_t dx = (int64_t)o.x - p.x, dy = (int64_t)o.y - p.y, dz = (int64_t)o.z - p.z;
        // grown balls meet only within 2h <= 2^13 quanta per axis
        const int64_t lim = 1 << 20;
        if (dx >= lim || dx <= -lim || dy >= lim || dy <= -lim || dz >= lim || dz <= -lim) return false;
        if (dx == 0 && dy == 0 && dz == 0) {
            atomicOr(&cnt->err, DERR_COINCIDENT);
            return false;
        }
        const int64_t sx = (int64_t)o.w + pc.A;
        return sx >= 0 && grown_meet(dx * dx + dy * dy + dz * dz, si, sx);
    }
}

template <int MODE, bool SMALL>
__global__ void __launch_bounds__(NB_THREADS)
    k_neighbours(const int4* __restrict__ Ps, const int32_t* __restrict__ mol_s, const MolGrid* __restrict__ grids,
                 const uint32_t* __restrict__ cell_start, PredConst pc, int64_t n, int64_t* __restrict__ nb_cnt,
                 const int64_t* __restrict__ nb_off, int32_t* __restrict__ nb, DevCounters* __restrict__ cnt,
                 int64_t* __restrict__ pw) {
    const int64_t s = (int64_t)blockIdx.x * NB_THREADS + threadIdx.x;
    int64_t count = 0;
    if (s < n) {
        const int4 p = Ps[s];
        const int64_t si = (int64_t)p.w + pc.A;
        const int64_t w = MODE == NB_CSR ? nb_off[s] : MODE == NB_PADDED ? s * NB_STRIDE : 0;
        if (si >= 0) {
            const MolGrid g = grids[mol_s[s]];
            const int cell = pc.cell, R = pc.reach;
            const int cx = (p.x - g.org[0]) / cell, cy = (p.y - g.org[1]) / cell, cz = (p.z - g.org[2]) / cell;
            const int z0 = max(cz - R, 0), z1 = min(cz + R, g.dims[2] - 1);
            const int y0 = max(cy - R, 0), y1 = min(cy + R, g.dims[1] - 1);
            const int x0 = max(cx - R, 0), x1 = min(cx + R, g.dims[0] - 1);
            const int32_t si32 = (int32_t)si;  // W + A <= 2^24
            const int A32 = (int)max(pc.A, -(int64_t)(1 << 30));  // below -2^24 no grown ball exists
            for (int z = z0; z <= z1; z++)
                for (int y = y0; y <= y1; y++) {
                    const int64_t row = g.cell_base + ((int64_t)z * g.dims[1] + y) * g.dims[0];
                    const uint32_t a = cell_start[row + x0], b = cell_start[row + x1 + 1];
                    for (uint32_t t0 = a; t0 < b; t0 += NB_UNROLL) {
                        int4 ov[NB_UNROLL];
#pragma unroll
                        for (int u = 0; u < NB_UNROLL; u++) ov[u] = __ldg(&Ps[t0 + u < b ? t0 + u : a]);
#pragma unroll
                        for (int u = 0; u < NB_UNROLL; u++) {
                            const uint32_t t = t0 + u;
                            if (t < b && t != (uint32_t)s && nb_meet<SMALL>(p, si, si32, A32, pc, ov[u], cnt)) {
                                if (MODE == NB_CSR || (MODE == NB_PADDED && count < NB_STRIDE)) nb[w + count] = (int32_t)t;
                                count++;
                            }
                        }
                    }
                }
        }
        if (MODE != NB_CSR) {
            nb_cnt[s] = count;
            pw[s] = pair_mask_words((int)count);  // the K^2 pair mask of this atom
        }
    }
    if (MODE != NB_CSR) {
        // one pair of atomics per block; every thread reaches here (no early exit above)
        __shared__ unsigned long long b_tot[NB_THREADS / 32];
        __shared__ int b_max[NB_THREADS / 32];
        const unsigned wt = __reduce_add_sync(0xffffffffu, (unsigned)count);
        const unsigned wm = __reduce_max_sync(0xffffffffu, (unsigned)count);
        if ((threadIdx.x & 31) == 0) {
            b_tot[threadIdx.x >> 5] = wt;
            b_max[threadIdx.x >> 5] = (int)wm;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            unsigned long long tot = 0;
            int m = 0;
            for (int k = 0; k < NB_THREADS / 32; k++) {
                tot += b_tot[k];
                m = max(m, b_max[k]);
            }
            if (tot) atomicAdd(&cnt->nb_sum, tot);
            atomicMax(&cnt->max_degree, m);
        }
    }
}

// Blocks of k_neighbours: one thread per atom.
static unsigned neighbour_blocks(int64_t n) { return (unsigned)((n + NB_THREADS - 1) / NB_THREADS); }

// Work order of the per-atom pass: sorted positions by decreasing neighbour
// count (ties in any order), so the costliest atoms start first and the
// kernel's tail is short; the atoms with more than 64 neighbours form its head.
constexpr int DEG_BINS = 259;  // counts 0..256, 257 for 257..512, 258 for anything above

__device__ __forceinline__ int deg_bin(int64_t m) { return m > 512 ? 258 : m > 256 ? 257 : (int)m; }

__global__ void k_deg_hist(const int64_t* __restrict__ cnt, int64_t n, unsigned* __restrict__ hist) {
    __shared__ unsigned h[DEG_BINS];
    for (int t = threadIdx.x; t < DEG_BINS; t += blockDim.x) h[t] = 0;
    __syncthreads();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) atomicAdd(&h[deg_bin(cnt[i])], 1u);
    __syncthreads();
    for (int t = threadIdx.x; t < DEG_BINS; t += blockDim.x)
        if (h[t]) atomicAdd(&hist[t], h[t]);
}

// start of each bin in decreasing order, and the head sizes (atoms with more
// than 64, and more than 512, neighbours): one thread per bin
__global__ void k_deg_starts(const unsigned* __restrict__ hist, unsigned* __restrict__ cursor,
                             long long* __restrict__ n_wide) {
    __shared__ unsigned h[DEG_BINS];
    const int b = threadIdx.x;
    if (b < DEG_BINS) h[b] = hist[b];
    __syncthreads();
    if (b >= DEG_BINS) return;
    unsigned run = 0;
    for (int q = DEG_BINS - 1; q > b; q--) run += h[q];
    cursor[b] = run;
    // atoms over 64, 512, 128 and 256 neighbours: the tiers of the per-atom pass
    if (b == 65) n_wide[0] = run + h[65];
    if (b == DEG_BINS - 1) n_wide[1] = h[DEG_BINS - 1];
    if (b == 129) n_wide[2] = run + h[129];
    if (b == DEG_BINS - 2) n_wide[3] = run + h[DEG_BINS - 2];
}

__global__ void k_deg_scatter(const int64_t* __restrict__ cnt, int64_t n, unsigned* __restrict__ cursor,
                              int32_t* __restrict__ work) {
    __shared__ unsigned h[DEG_BINS], base[DEG_BINS];
    for (int t = threadIdx.x; t < DEG_BINS; t += blockDim.x) h[t] = 0;
    __syncthreads();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int b = i < n ? deg_bin(cnt[i]) : 0;
    const unsigned local = i < n ? atomicAdd(&h[b], 1u) : 0u;
    __syncthreads();
    for (int t = threadIdx.x; t < DEG_BINS; t += blockDim.x)
        if (h[t]) base[t] = atomicAdd(&cursor[t], h[t]);
    __syncthreads();
    if (i < n) work[base[b] + local] = (int32_t)i;
}

// L(i) for every atom. With at most NB_STRIDE neighbours per atom (always so
// for atomic radii and a 1.4 A probe) one pass counts and writes padded rows;
// otherwise the counts are scanned into offsets and a second pass writes the
// compact lists. The work order of the per-atom pass comes from the counts.
int build_neighbours(ac_ctx* c, cudaStream_t s) {
    const int64_t n = c->n;
    AC_TRY(c->nb_cnt.reserve((size_t)(n + 1) * sizeof(int64_t), s));
    int64_t* cntp = c->nb_cnt.as<int64_t>();
    if (n == 0) {
        c->nb_total = 0;
        c->n_wide = c->n_huge = c->n_w128 = c->n_w256 = 0;
        c->nb_stride = 0;
        c->pair_words = 0;
        AC_CUDA(cudaMemsetAsync(cntp, 0, sizeof(int64_t), s));
        AC_TRY(c->nb.reserve(4, s));
        return AC_OK;
    }
    const unsigned nb = (unsigned)((n + 127) / 128);
    DevCounters* dc = c->counters.as<DevCounters>();
    const bool small = (int64_t)(c->pc.reach + 1) * c->pc.cell < NB_SPAN_SMALL;
    const unsigned kb = neighbour_blocks(n);
    // a replay keeps the recorded layout; a synchronised build tries the padded one
    const bool padded = c->replaying ? c->rec.nb_stride == NB_STRIDE : true;
    const GridView g{c->Ps.as<int4>(), c->mol_s.as<int32_t>(), c->grids.as<MolGrid>(), c->cell_start.as<uint32_t>()};
    AC_TRY(c->cw.cnt.reserve((size_t)(n + 1) * sizeof(int64_t), s));
    int64_t* pw = c->cw.cnt.as<int64_t>();
    if (padded) {
        AC_TRY(c->nb.reserve((size_t)n * NB_STRIDE * sizeof(int32_t), s));
        auto k = small ? k_neighbours<NB_PADDED, true> : k_neighbours<NB_PADDED, false>;
        k<<<kb, NB_THREADS, 0, s>>>(g.Ps, g.mol_s, g.grids, g.cell_start, c->pc, n, cntp, nullptr, c->nb.as<int32_t>(), dc, pw);
    } else {
        auto k = small ? k_neighbours<NB_COUNT, true> : k_neighbours<NB_COUNT, false>;
        k<<<kb, NB_THREADS, 0, s>>>(g.Ps, g.mol_s, g.grids, g.cell_start, c->pc, n, cntp, nullptr, nullptr, dc, pw);
    }
    AC_LAUNCHED();
    // layout of the K^2 pair masks, from the words per atom
    AC_TRY(plan_pair_masks(c, pw, s));
    // work order from the counts (before a scan turns them into offsets)
    AC_TRY(c->work.reserve((size_t)n * sizeof(int32_t), s));
    AC_TRY(c->deg.reserve(2 * DEG_BINS * sizeof(unsigned) + 64, s));
    unsigned* hist = c->deg.as<unsigned>();
    unsigned* cursor = hist + DEG_BINS;
    static_assert((2 * DEG_BINS * sizeof(unsigned)) % 8 == 0, "head counts 8-aligned");
    // atoms over 64 neighbours, over 512 (n_huge), over 128, over 256
    long long* n_wide = reinterpret_cast<long long*>(hist + 2 * DEG_BINS);
    AC_CUDA(cudaMemsetAsync(hist, 0, DEG_BINS * sizeof(unsigned), s));
    k_deg_hist<<<nb, 128, 0, s>>>(cntp, n, hist);
    AC_LAUNCHED();
    k_deg_starts<<<1, (DEG_BINS + 31) / 32 * 32, 0, s>>>(hist, cursor, n_wide);
    AC_LAUNCHED();
    k_deg_scatter<<<nb, 128, 0, s>>>(cntp, n, cursor, c->work.as<int32_t>());
    AC_LAUNCHED();
    int64_t total = 0;
    bool compact = !padded;
    if (c->replaying) {
        // sizes of the recorded build, checked on the device
        total = c->rec.nb_total;
        c->n_wide = c->rec.n_wide;
        c->n_huge = c->rec.n_huge;
        c->n_w128 = c->rec.n_w128;
        c->n_w256 = c->rec.n_w256;
        AC_TRY(expect_u64(c, &dc->nb_sum, (unsigned long long)total, s));
        AC_TRY(expect_i64(c, reinterpret_cast<const int64_t*>(n_wide), c->n_wide, s));
        AC_TRY(expect_i64(c, reinterpret_cast<const int64_t*>(n_wide + 1), c->n_huge, s));
        AC_TRY(expect_i64(c, reinterpret_cast<const int64_t*>(n_wide + 2), c->n_w128, s));
        AC_TRY(expect_i64(c, reinterpret_cast<const int64_t*>(n_wide + 3), c->n_w256, s));
        AC_TRY(expect_i64(c, c->pair_moff.as<int64_t>() + n, c->pair_words, s));
    } else {
        AC_CUDA(cudaMemcpyAsync(c->h_stage + 1, n_wide, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        AC_CUDA(cudaMemcpyAsync(c->h_stage + 3, n_wide + 1, 3 * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        AC_CUDA(cudaMemcpyAsync(c->h_stage + 2, c->pair_moff.as<int64_t>() + n, sizeof(int64_t),
                                cudaMemcpyDeviceToHost, s));
        DevCounters h;
        AC_TRY(read_counters(c, &h, s));  // also completes the copies above
        total = (int64_t)h.nb_sum;
        c->n_wide = c->h_stage[1];
        c->n_huge = c->h_stage[3];
        c->n_w128 = c->h_stage[4];
        c->n_w256 = c->h_stage[5];
        c->pair_words = c->h_stage[2];
        if (h.err & DERR_COINCIDENT)
            return fail(AC_ERR_DEGENERATE, "two centres coincide after quantisation to 1/1024 A");
        if (h.max_degree > NB_STRIDE) compact = true;  // rows too short: redo as compact lists
    }
    c->nb_total = total;
    c->nb_stride = compact ? 0 : NB_STRIDE;
    if (!compact) return AC_OK;
    AC_TRY(scan_exclusive_i64(c, cntp, cntp, n, s));
    if (c->replaying) AC_TRY(expect_i64(c, cntp + n, total, s));
    AC_TRY(c->nb.reserve((size_t)(total > 0 ? total : 1) * sizeof(int32_t), s));
    auto k_fill = small ? k_neighbours<NB_CSR, true> : k_neighbours<NB_CSR, false>;
    k_fill<<<kb, NB_THREADS, 0, s>>>(g.Ps, g.mol_s, g.grids, g.cell_start, c->pc, n, nullptr, cntp, c->nb.as<int32_t>(), dc,
                              nullptr);
    AC_LAUNCHED();
    return AC_OK;
}

}  // namespace ac
