/*
 * Seeded synthetic atom sets that stand in for the biomolecules of the
 * paper's experiments (Section 5: proteins of 10^3..10^5 atoms and capsids of
 * ~6 M atoms, van der Waals radii, alpha in [0, 2]).
 *
 * This file holds only input generation: no geometry of the alpha-complex
 * method lives here. Both the CUDA path and the CPU oracle consume its output.
 *
 * Recipe (Section 4.1 lists the three properties it mimics: bounded radii,
 * a minimum centre separation, small alpha):
 *   - PRNG: xoshiro256** whose 256-bit state is filled by SplitMix64 from a
 *     64-bit seed; a uniform double is (next() >> 11) * 2^-53.
 *   - Random sequential addition: draw a point uniformly in the cube
 *     [-R_out, R_out]^3 (three uniforms, x then y then z); keep it if it lies in
 *     the region (ball |x| <= R_out, or shell R_in <= |x| <= R_out, tested in
 *     double); quantise each coordinate to X = round_half_even(1024 x); reject
 *     it if an accepted centre lies at integer squared distance < MIN_SEP2
 *     quanta^2 (1.3 A separation); otherwise accept it and draw one more
 *     uniform u for the element: C if u < .63, N if u < .80, O if u < .99,
 *     else S.
 *   - Radii are quantised per element (1/1024 A units, round half even):
 *     van der Waals C 1741, N 1587, O 1556, S 1843; with the 1.4 A solvent
 *     probe added first: C 3174, N 3021, O 2990, S 3277.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

#define MIN_SEP2 1772094LL /* ceil((1.3 * 1024)^2) */

typedef struct { uint64_t s[4]; } xo256;

static uint64_t splitmix64(uint64_t *x) {
    uint64_t z = (*x += 0x9e3779b97f4a7c15ULL);
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

static uint64_t rotl(uint64_t x, int k) { return (x << k) | (x >> (64 - k)); }

static uint64_t xo_next(xo256 *g) {
    uint64_t *s = g->s;
    uint64_t result = rotl(s[1] * 5, 7) * 9;
    uint64_t t = s[1] << 17;
    s[2] ^= s[0];
    s[3] ^= s[1];
    s[1] ^= s[2];
    s[0] ^= s[3];
    s[2] ^= t;
    s[3] = rotl(s[3], 45);
    return result;
}

static void xo_seed(xo256 *g, uint64_t seed) {
    uint64_t x = seed;
    for (int i = 0; i < 4; i++) g->s[i] = splitmix64(&x);
}

static double xo_uniform(xo256 *g) { return (double)(xo_next(g) >> 11) * 0x1.0p-53; }

/* Radii in quanta per element index (0 C, 1 N, 2 O, 3 S). */
static const int32_t RADIUS_VDW[4] = {1741, 1587, 1556, 1843};
static const int32_t RADIUS_PROBE[4] = {3174, 3021, 2990, 3277};

/* Open-addressing hash of occupied 1.3 A cells -> head of a per-atom chain. */
typedef struct {
    int64_t *keys;
    int32_t *head;
    uint64_t mask;
} cellhash;

static uint64_t mix_key(int64_t k) {
    uint64_t z = (uint64_t)k * 0x9e3779b97f4a7c15ULL;
    return z ^ (z >> 29);
}

static int64_t cell_key(int64_t cx, int64_t cy, int64_t cz) {
    return ((cx + (1 << 20)) << 42) | ((cy + (1 << 20)) << 21) | (cz + (1 << 20));
}

static int32_t *hash_slot(cellhash *h, int64_t key, int insert) {
    uint64_t i = mix_key(key) & h->mask;
    for (;;) {
        if (h->head[i] == -1) {
            if (!insert) return NULL;
            h->keys[i] = key;
            return &h->head[i];
        }
        if (h->keys[i] == key) return &h->head[i];
        i = (i + 1) & h->mask;
    }
}

/*
 * Generate n centres (quantised ints, n x 3) and radii (quantised ints) and
 * element codes. r_in < 0 means a full ball of radius r_out.
 * Returns 0 on success, -1 on allocation failure, -2 if the region cannot
 * hold n atoms within max_attempts draws.
 */
int synth_atoms(uint64_t seed, int64_t n, double r_in, double r_out, int probe,
                int32_t *xyz, int32_t *radius, uint8_t *element) {
    if (n <= 0) return 0;
    const int64_t cell = 1332; /* >= 1.3 A in quanta, so a 27-cell scan suffices */
    uint64_t cap = 1;
    while (cap < (uint64_t)(4 * n)) cap <<= 1;
    cellhash h;
    h.mask = cap - 1;
    h.keys = (int64_t *)malloc(cap * sizeof(int64_t));
    h.head = (int32_t *)malloc(cap * sizeof(int32_t));
    int32_t *next = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    if (!h.keys || !h.head || !next) {
        free(h.keys); free(h.head); free(next);
        return -1;
    }
    memset(h.head, 0xff, cap * sizeof(int32_t));
    xo256 g;
    xo_seed(&g, seed);
    const int32_t *rad = probe ? RADIUS_PROBE : RADIUS_VDW;
    int64_t accepted = 0;
    int64_t attempts = 0, max_attempts = 2000 * n + 1000000;
    double r_in2 = r_in > 0 ? r_in * r_in : -1.0, r_out2 = r_out * r_out;
    while (accepted < n) {
        if (++attempts > max_attempts) {
            free(h.keys); free(h.head); free(next);
            return -2;
        }
        double x = (2.0 * xo_uniform(&g) - 1.0) * r_out;
        double y = (2.0 * xo_uniform(&g) - 1.0) * r_out;
        double z = (2.0 * xo_uniform(&g) - 1.0) * r_out;
        double d2 = x * x + y * y + z * z;
        if (d2 > r_out2 || d2 < r_in2) continue;
        int64_t X = (int64_t)nearbyint(1024.0 * x);
        int64_t Y = (int64_t)nearbyint(1024.0 * y);
        int64_t Z = (int64_t)nearbyint(1024.0 * z);
        int64_t cx = (int64_t)floor((double)X / cell), cy = (int64_t)floor((double)Y / cell),
                cz = (int64_t)floor((double)Z / cell);
        int clash = 0;
        for (int dz = -1; dz <= 1 && !clash; dz++)
            for (int dy = -1; dy <= 1 && !clash; dy++)
                for (int dx = -1; dx <= 1 && !clash; dx++) {
                    int32_t *hd = hash_slot(&h, cell_key(cx + dx, cy + dy, cz + dz), 0);
                    if (!hd) continue;
                    for (int32_t a = *hd; a != -1; a = next[a]) {
                        int64_t ex = X - xyz[3 * a], ey = Y - xyz[3 * a + 1], ez = Z - xyz[3 * a + 2];
                        if (ex * ex + ey * ey + ez * ez < MIN_SEP2) { clash = 1; break; }
                    }
                }
        if (clash) continue;
        xyz[3 * accepted] = (int32_t)X;
        xyz[3 * accepted + 1] = (int32_t)Y;
        xyz[3 * accepted + 2] = (int32_t)Z;
        int32_t *hd = hash_slot(&h, cell_key(cx, cy, cz), 1);
        next[accepted] = *hd;
        *hd = (int32_t)accepted;
        double u = xo_uniform(&g);
        int e = u < 0.63 ? 0 : (u < 0.80 ? 1 : (u < 0.99 ? 2 : 3));
        element[accepted] = (uint8_t)e;
        radius[accepted] = rad[e];
        accepted++;
    }
    free(h.keys); free(h.head); free(next);
    return 0;
}

/* Molecule sizes for a batch: log-uniform in [lo, hi], rounded half even. */
void synth_batch_sizes(uint64_t seed, int64_t n_mol, double lo, double hi, int64_t *sizes) {
    xo256 g;
    xo_seed(&g, seed);
    double a = log(lo), b = log(hi);
    for (int64_t m = 0; m < n_mol; m++) sizes[m] = (int64_t)nearbyint(exp(a + (b - a) * xo_uniform(&g)));
}

/* Standard normal draws (Box-Muller on two uniforms), used for loss weights. */
void synth_normal(uint64_t seed, int64_t n, double *out) {
    xo256 g;
    xo_seed(&g, seed);
    for (int64_t i = 0; i < n; i += 2) {
        double u1 = 1.0 - xo_uniform(&g), u2 = xo_uniform(&g);
        double r = sqrt(-2.0 * log(u1)), t = 6.283185307179586 * u2;
        out[i] = r * cos(t);
        if (i + 1 < n) out[i + 1] = r * sin(t);
    }
}

/* The first k raw outputs for a seed (for the generator's own test). */
void synth_raw(uint64_t seed, int64_t k, uint64_t *out) {
    xo256 g;
    xo_seed(&g, seed);
    for (int64_t i = 0; i < k; i++) out[i] = xo_next(&g);
}
