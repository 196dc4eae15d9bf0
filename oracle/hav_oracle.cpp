// HAVSampler CPU oracle -- TEST INFRASTRUCTURE ONLY.
//
// A plain, slow, single-threaded restatement of the hierarchical adaptive
// voxel-guided sampler (arXiv 2305.14306, Section 3).  It exists to check the
// CUDA path; it is never part of it.  Only the test suite, the smoke check
// and the benchmark's CPU-baseline leg may load it.  It shares no code, no
// header and no constant table with the CUDA library: every definition below
// is written out here on its own.
//
// Build: g++ -std=c++17 -O2 -ffp-contract=off -fno-fast-math -fPIC -shared
// (-ffp-contract=off matters: the voxel keys and centre distances must be
// plain IEEE-754 binary32 operations rounded to nearest, with no fused
// multiply-add, so that the result is defined by the arithmetic alone.)
//
// Readings of the paper fixed here (each one is a choice the text leaves open):
//   * Eq. 2 grid anchored at the origin; keys are made relative to the
//     bounding-box minimum cell so they pack into 3 x 21 bits.
//   * The voxel vector is v = s * r for a scalar s searched by bisection over
//     (0, s_hi], s_hi = max_a (E_a / r_a), E_a the bounding-box extent.
//   * Section 3.3 stopping rule: accept when m <= K <= m + floor(m*sigma).
//     Without acceptance after t_max steps: s* = lo if lo > 0 (truncate),
//     otherwise s* = hi (shortfall fill).
//   * Section 3.2 centre-closest rule uses the squared distance; ties on the
//     squared distance go to the lowest point index.
//   * "cut off" (Section 3.3) is a deterministic truncation: keep the m_l
//     voxels whose SplitMix64-finalised key is smallest.
//   * Eq. 3 layer budgets with ratio 4: m_l = floor(m * 4^(l-1) / S) for the
//     first k-1 layers, the last layer takes the remainder, S = sum 4^(l-1).
//   * Output is every taken index in ascending order.
//   * Section 3.3 search, "guided" mode (search = 1; the default search = 0 is
//     the bisection above): the paper bounds the search by ceil(log 1/sigma)
//     steps, which needs a starting bracket near s*.  After the first search
//     of a call (per cloud, across layers and levels) the next search starts
//     from g = s_prev * sqrt(m_prev / m_l): the previous search's s* and budget
//     under the surface law K ~ s^-2.  While every count so far exceeded
//     k_max, the next size is 2 * lo (doubling up from g) as long as that stays
//     below hi; otherwise, and after the first count below m_l, it is the
//     bisection midpoint.  g >= s_hi, or no previous search, gives the plain
//     bisection.
//   * Table 6 variants (Section 4.5): RA keeps, per voxel, the point with the
//     smallest counter-based SplitMix64 draw (seed, index); ME and CE keep the
//     centre-closest index and report the voxel's mean (fixed-point sums, see
//     voxel_mean) or centre v * (g + 0.5); a fixed voxel size skips the search.
//
// Parity: the voxel grouping, the centre-closest argmin, Cnt, the bisection
// trace and the layer recursion are pinned by tests that do not call this
// file's arithmetic (brute-force grouping in numpy, closed-form lattice
// counts, nested-grid monotonicity, hand-built cases, permutation checks).

#include <cmath>
#include <cstdint>
#include <cstring>
#include <algorithm>
#include <unordered_map>
#include <unordered_set>
#include <vector>

namespace {

enum {
    OR_SEL_CC = 0,
    OR_SEL_RA = 1,
    OR_SEL_ME = 2,
    OR_SEL_CE = 3,
};

enum {
    OR_OK = 0,
    OR_ERR_INVALID = 1,
    OR_ERR_NONFINITE = 2,
    OR_ERR_RANGE = 7,
};

constexpr int kAxisBits = 21;
constexpr int64_t kAxisLimit = int64_t(1) << kAxisBits;
constexpr int kMaxIters = 20;

}  // namespace

extern "C" {

// The oracle's own parameter block (the CUDA library declares its own).
typedef struct {
    int32_t sigma_num;    // tolerance sigma = sigma_num / sigma_den (0.05)
    int32_t sigma_den;
    int32_t t_max;        // bisection steps, 0..20 (20)
    int32_t layers;       // k, >= 1 (2)
    int32_t layer_ratio;  // m_l = ratio * m_(l-1) (4)
    float aspect[3];      // r, v = s * r (1, 1, 1)
    uint32_t flags;       // unused, must be 0
    int32_t select;       // 0 centre-closest, 1 random, 2 mean, 3 centre (Table 6)
    uint32_t seed;        // draws of the random selection
    float fixed_s;        // > 0: fixed voxel size s (no search); 0: adaptive
    int32_t search;       // 0 bisection over (0, s_hi]; 1 guided by the previous search
} hor_params;

// Per-layer record of one call: what the bisection evaluated and decided.
typedef struct {
    int64_t m_l;           // this layer's budget
    int64_t k_max;         // m_l + floor(m_l * sigma)
    int64_t k_star;        // occupied voxels at the chosen s*
    int64_t n_in;          // untaken points entering the layer
    int32_t iters;         // bisection steps evaluated
    int32_t accepted;      // 1 if a step landed in [m_l, k_max]
    float s_hi;            // top of the search bracket
    float s_star;          // chosen scalar voxel size
    float s[kMaxIters];    // evaluated s per step
    int64_t K[kMaxIters];  // Cnt at that s (exact)
} hor_layer_trace;

}  // extern "C"

namespace {

struct Ctx {
    float mn[3];
    float s_hi;
    float r[3];
};

// The previous search of this cloud within one call (guided search mode).
struct Guide {
    bool valid = false;
    float s = 0.0f;     // its chosen s*
    int64_t m = 0;      // its budget m_l
};

// Eq. 2: g_a = floor(x_a / v_a), then made relative to the cell of the
// bounding-box minimum.  Returns false when a cell index leaves the packable
// range (or the quotient is not a usable integer).
bool floor_div(float x, float v, int64_t* F, float* f_out) {
    float q = x / v;
    float f = std::floor(q);
    if (!(std::fabs(f) < 4.6e18f)) return false;  // |f| < 2^62, excludes inf/nan
    *F = static_cast<int64_t>(f);
    if (f_out) *f_out = f;
    return true;
}

bool voxel_size(const Ctx& c, float s, float v[3]) {
    for (int a = 0; a < 3; ++a) {
        v[a] = s * c.r[a];
        if (!(v[a] > 0.0f) || !std::isfinite(v[a])) return false;
    }
    return true;
}

bool min_cells(const Ctx& c, const float v[3], int64_t fmin[3]) {
    for (int a = 0; a < 3; ++a)
        if (!floor_div(c.mn[a], v[a], &fmin[a], nullptr)) return false;
    return true;
}

bool voxel_key(const float* p, const float v[3], const int64_t fmin[3],
               uint64_t* key, float f[3]) {
    uint64_t k = 0;
    for (int a = 0; a < 3; ++a) {
        int64_t F;
        if (!floor_div(p[a], v[a], &F, &f[a])) return false;
        int64_t u = F - fmin[a];
        if (u < 0 || u >= kAxisLimit) return false;
        k |= static_cast<uint64_t>(u) << (kAxisBits * a);
    }
    *key = k;
    return true;
}

// Section 3.2: squared distance of the point to its voxel centre
// v * (g + 0.5), binary32, fixed order, no fusion.
float centre_dist2(const float* p, const float v[3], const float f[3]) {
    float d[3];
    for (int a = 0; a < 3; ++a) {
        float half = f[a] + 0.5f;
        float centre = v[a] * half;
        d[a] = p[a] - centre;
    }
    float xx = d[0] * d[0];
    float yy = d[1] * d[1];
    float zz = d[2] * d[2];
    float xy = xx + yy;
    return xy + zz;
}

uint32_t float_bits(float x) {
    uint32_t b;
    std::memcpy(&b, &x, 4);
    return b;
}

// SplitMix64 output finaliser (Steele, Lea, Flood 2014): a bijection on
// 64-bit words, used as the truncation priority of a voxel key.
uint64_t splitmix_finalise(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Counter-based draw number `counter` of the SplitMix64 generator started at
// `seed` (Steele, Lea, Flood 2014): the state after counter + 1 increments of
// the golden-ratio step, finalised.
uint64_t random_draw(uint32_t seed, uint64_t counter) {
    const uint64_t z = static_cast<uint64_t>(seed) + (counter + 1) * 0x9E3779B97F4A7C15ull;
    return splitmix_finalise(z);
}

// Cnt(P_l, s) of Section 3.3: number of distinct voxel keys among the points
// listed in `active`.
int count_voxels(const float* pts, const std::vector<int32_t>& active,
                 const Ctx& c, float s, int64_t* K) {
    float v[3];
    int64_t fmin[3];
    if (!voxel_size(c, s, v) || !min_cells(c, v, fmin)) return OR_ERR_RANGE;
    std::unordered_set<uint64_t> seen;
    seen.reserve(active.size() * 2 + 1);
    for (int32_t i : active) {
        uint64_t key;
        float f[3];
        if (!voxel_key(pts + 3 * int64_t(i), v, fmin, &key, f)) return OR_ERR_RANGE;
        seen.insert(key);
    }
    *K = static_cast<int64_t>(seen.size());
    return OR_OK;
}

int bounding_box(const float* pts, int64_t n, const float r[3], Ctx* c) {
    float mn[3], mx[3];
    for (int a = 0; a < 3; ++a) { mn[a] = INFINITY; mx[a] = -INFINITY; }
    for (int64_t i = 0; i < n; ++i)
        for (int a = 0; a < 3; ++a) {
            float x = pts[3 * i + a];
            if (!std::isfinite(x)) return OR_ERR_NONFINITE;
            mn[a] = std::min(mn[a], x);
            mx[a] = std::max(mx[a], x);
        }
    float s_hi = 0.0f;
    for (int a = 0; a < 3; ++a) {
        float e = mx[a] - mn[a];
        float t = e / r[a];
        s_hi = std::max(s_hi, t);
        c->mn[a] = mn[a];
        c->r[a] = r[a];
    }
    if (n == 0 || s_hi == 0.0f) s_hi = 1.0f;  // all points coincide: K = 1 for any s
    if (!std::isfinite(s_hi)) return OR_ERR_RANGE;
    c->s_hi = s_hi;
    return OR_OK;
}

int check_params(const hor_params* p) {
    if (!p) return OR_ERR_INVALID;
    if (p->sigma_num < 0 || p->sigma_den <= 0) return OR_ERR_INVALID;
    if (p->t_max < 0 || p->t_max > kMaxIters) return OR_ERR_INVALID;
    if (p->layers < 1 || p->layers > 8) return OR_ERR_INVALID;
    if (p->layer_ratio < 1 || p->layer_ratio > 64) return OR_ERR_INVALID;
    for (int a = 0; a < 3; ++a)
        if (!(p->aspect[a] > 0.0f) || !std::isfinite(p->aspect[a])) return OR_ERR_INVALID;
    if (p->flags != 0) return OR_ERR_INVALID;
    if (p->select < OR_SEL_CC || p->select > OR_SEL_CE) return OR_ERR_INVALID;
    if (p->search != 0 && p->search != 1) return OR_ERR_INVALID;
    if (!(p->fixed_s >= 0.0f) || !std::isfinite(p->fixed_s)) return OR_ERR_INVALID;
    // the ablation variants run one layer, as in Table 6
    if ((p->fixed_s > 0.0f || p->select == OR_SEL_ME || p->select == OR_SEL_CE) && p->layers != 1)
        return OR_ERR_INVALID;
    return OR_OK;
}

// Eq. 3 budgets: m_l = 4 m_(l-1) and sum m_l = m.
std::vector<int64_t> layer_budgets(int64_t m, int layers, int ratio) {
    std::vector<int64_t> w(layers);
    int64_t S = 0, pw = 1;
    for (int l = 0; l < layers; ++l) { w[l] = pw; S += pw; pw *= ratio; }
    std::vector<int64_t> ml(layers);
    int64_t used = 0;
    for (int l = 0; l + 1 < layers; ++l) {
        ml[l] = (m * w[l]) / S;
        used += ml[l];
    }
    ml[layers - 1] = m - used;
    return ml;
}

// One HAVSampler call on pts[0..n): fills taken[] and the trace; `guide`
// carries the previous search of the cloud (guided search mode).
int sample_one(const float* pts, int64_t n, int64_t m, const hor_params* p,
               std::vector<uint8_t>& taken, hor_layer_trace* tr, Guide* guide) {
    Ctx c;
    int st = bounding_box(pts, n, p->aspect, &c);
    if (st != OR_OK) return st;
    taken.assign(static_cast<size_t>(n), 0);
    std::vector<int64_t> ml = layer_budgets(m, p->layers, p->layer_ratio);

    for (int l = 0; l < p->layers; ++l) {
        hor_layer_trace rec;
        std::memset(&rec, 0, sizeof rec);
        const int64_t m_l = ml[l];
        const int64_t k_max = m_l + (m_l * p->sigma_num) / p->sigma_den;
        rec.m_l = m_l;
        rec.k_max = k_max;
        rec.s_hi = c.s_hi;
        if (m_l == 0) {
            if (tr) tr[l] = rec;
            continue;
        }
        // P_l: the points not taken by coarser layers, ascending.
        std::vector<int32_t> active;
        for (int64_t i = 0; i < n; ++i)
            if (!taken[i]) active.push_back(static_cast<int32_t>(i));
        rec.n_in = static_cast<int64_t>(active.size());

        // Section 3.3 adaptive voxel search (skipped for a fixed voxel size).
        float lo = 0.0f, hi = c.s_hi, s_star = 0.0f;
        bool accepted = false;
        const bool fixed = p->fixed_s > 0.0f;
        // guided mode: start at g and double while the counts stay above k_max
        float first = 0.0f;
        bool up = false;
        if (p->search == 1) {
            float g;
            if (guide->valid) {
                const float ratio = static_cast<float>(guide->m) / static_cast<float>(m_l);
                g = guide->s * std::sqrt(ratio);
            } else {
                g = c.s_hi / std::sqrt(static_cast<float>(m_l));
            }
            if (g > 0.0f && g < hi) {
                first = g;
                up = true;
            }
        }
        for (int t = 0; t < (fixed ? 0 : p->t_max); ++t) {
            float s;
            if (t == 0 && first > 0.0f) s = first;
            else if (up && lo * 2.0f < hi) s = lo * 2.0f;
            else s = (lo + hi) * 0.5f;
            int64_t K;
            st = count_voxels(pts, active, c, s, &K);
            if (st != OR_OK) return st;
            rec.s[t] = s;
            rec.K[t] = K;
            rec.iters = t + 1;
            if (K > k_max) {
                lo = s;
            } else if (K < m_l) {
                hi = s;
                up = false;
            } else {
                s_star = s;
                accepted = true;
                break;
            }
        }
        if (!accepted) s_star = (lo > 0.0f) ? lo : hi;
        if (fixed) s_star = p->fixed_s;
        if (!fixed && p->t_max > 0) {
            guide->valid = true;
            guide->s = s_star;
            guide->m = m_l;
        }
        rec.accepted = accepted ? 1 : 0;
        rec.s_star = s_star;

        // Section 3.2 centre-closest selection at s*.
        float v[3];
        int64_t fmin[3];
        if (!voxel_size(c, s_star, v) || !min_cells(c, v, fmin)) return OR_ERR_RANGE;
        std::unordered_map<uint64_t, uint64_t> table;
        table.reserve(active.size() * 2 + 1);
        for (int32_t i : active) {
            uint64_t key;
            float f[3];
            const float* pi = pts + 3 * int64_t(i);
            if (!voxel_key(pi, v, fmin, &key, f)) return OR_ERR_RANGE;
            // the voxel's representative minimises this word: the squared
            // distance to the centre (CC, and ME / CE, which report other
            // coordinates for the same voxel) or a random draw (RA); ties
            // go to the lowest index
            uint32_t hi32;
            if (p->select == OR_SEL_RA) hi32 = static_cast<uint32_t>(random_draw(p->seed, uint64_t(i)) >> 32);
            else hi32 = float_bits(centre_dist2(pi, v, f));
            uint64_t packed = (static_cast<uint64_t>(hi32) << 32) | static_cast<uint32_t>(i);
            auto it = table.find(key);
            if (it == table.end()) table.emplace(key, packed);
            else if (packed < it->second) it->second = packed;
        }
        const int64_t K = static_cast<int64_t>(table.size());
        rec.k_star = K;

        std::vector<int32_t> reps;
        if (K > m_l) {
            // Cut off: keep the m_l voxels with the smallest priority.
            std::vector<std::pair<uint64_t, int32_t>> pr;
            pr.reserve(table.size());
            for (const auto& kv : table)
                pr.emplace_back(splitmix_finalise(kv.first),
                                static_cast<int32_t>(kv.second & 0xffffffffu));
            std::sort(pr.begin(), pr.end());
            for (int64_t j = 0; j < m_l; ++j) reps.push_back(pr[j].second);
        } else {
            for (const auto& kv : table)
                reps.push_back(static_cast<int32_t>(kv.second & 0xffffffffu));
        }
        for (int32_t i : reps) taken[i] = 1;
        if (K < m_l) {
            // Shortfall: untaken points in ascending index order.
            int64_t need = m_l - K;
            for (int32_t i : active) {
                if (need == 0) break;
                if (!taken[i]) { taken[i] = 1; --need; }
            }
        }
        if (tr) tr[l] = rec;
    }
    return OR_OK;
}

int sample_guided(const float* pts, int64_t n, int64_t m, const hor_params* p, int32_t* out,
                  hor_layer_trace* tr, Guide* guide) {
    int st = check_params(p);
    if (st != OR_OK) return st;
    if (n < 0 || m < 0 || m > n || n >= (int64_t(1) << 31)) return OR_ERR_INVALID;
    if (m == 0) return OR_OK;
    if (!pts || !out) return OR_ERR_INVALID;
    std::vector<uint8_t> taken;
    st = sample_one(pts, n, m, p, taken, tr, guide);
    if (st != OR_OK) return st;
    int64_t j = 0;
    for (int64_t i = 0; i < n; ++i)
        if (taken[i]) out[j++] = static_cast<int32_t>(i);
    return (j == m) ? OR_OK : OR_ERR_INVALID;
}

}  // namespace

extern "C" {

int hor_sample(const float* pts, int64_t n, int64_t m, const hor_params* p,
               int32_t* out, hor_layer_trace* tr) {
    Guide guide;
    return sample_guided(pts, n, m, p, out, tr, &guide);
}

// Level chain: level j+1 samples the points level j kept (in ascending
// order); every level's indices refer to the original cloud.
// out_concat holds level 0's m_levels[0] indices, then level 1's, ...
int hor_sample_levels(const float* pts, int64_t n, const int64_t* m_levels,
                      int32_t num_levels, const hor_params* p, int32_t* out_concat,
                      hor_layer_trace* tr) {
    int st = check_params(p);
    if (st != OR_OK) return st;
    if (num_levels < 1 || !m_levels) return OR_ERR_INVALID;
    if (n < 0 || n >= (int64_t(1) << 31)) return OR_ERR_INVALID;
    int64_t prev = n;
    for (int32_t j = 0; j < num_levels; ++j) {
        if (m_levels[j] < 0 || m_levels[j] > prev) return OR_ERR_INVALID;
        prev = m_levels[j];
    }
    std::vector<float> cur(pts, pts + 3 * n);
    std::vector<int32_t> orig(static_cast<size_t>(n));
    for (int64_t i = 0; i < n; ++i) orig[i] = static_cast<int32_t>(i);
    int64_t cur_n = n, off = 0;
    Guide guide;  // the guided search carries over from level to level
    for (int32_t j = 0; j < num_levels; ++j) {
        const int64_t m = m_levels[j];
        std::vector<int32_t> idx(static_cast<size_t>(m));
        if (m > 0) {
            st = sample_guided(cur.data(), cur_n, m, p, idx.data(),
                               tr ? tr + int64_t(j) * p->layers : nullptr, &guide);
            if (st != OR_OK) return st;
        }
        std::vector<float> nxt(static_cast<size_t>(3 * m));
        std::vector<int32_t> norig(static_cast<size_t>(m));
        for (int64_t r = 0; r < m; ++r) {
            const int32_t i = idx[r];
            for (int a = 0; a < 3; ++a) nxt[3 * r + a] = cur[3 * int64_t(i) + a];
            norig[r] = orig[i];
            out_concat[off + r] = orig[i];
        }
        off += m;
        cur.swap(nxt);
        orig.swap(norig);
        cur_n = m;
    }
    return OR_OK;
}

// Cnt(P, s) over all n points (bounding box taken from the same points).
int hor_count(const float* pts, int64_t n, float s, const float aspect[3], int64_t* K) {
    if (!pts || !K || n <= 0) return OR_ERR_INVALID;
    for (int a = 0; a < 3; ++a)
        if (!(aspect[a] > 0.0f) || !std::isfinite(aspect[a])) return OR_ERR_INVALID;
    Ctx c;
    int st = bounding_box(pts, n, aspect, &c);
    if (st != OR_OK) return st;
    std::vector<int32_t> all(static_cast<size_t>(n));
    for (int64_t i = 0; i < n; ++i) all[i] = static_cast<int32_t>(i);
    return count_voxels(pts, all, c, s, K);
}

// Packed voxel keys of every point at scalar size s (bounding box from pts).
int hor_keys(const float* pts, int64_t n, float s, const float aspect[3], uint64_t* keys) {
    if (!pts || !keys || n <= 0) return OR_ERR_INVALID;
    Ctx c;
    int st = bounding_box(pts, n, aspect, &c);
    if (st != OR_OK) return st;
    float v[3];
    int64_t fmin[3];
    if (!voxel_size(c, s, v) || !min_cells(c, v, fmin)) return OR_ERR_RANGE;
    for (int64_t i = 0; i < n; ++i) {
        float f[3];
        if (!voxel_key(pts + 3 * i, v, fmin, &keys[i], f)) return OR_ERR_RANGE;
    }
    return OR_OK;
}

// S(P, v) of Section 3.2 at a fixed scalar size s over all points: the
// centre-closest point of every occupied voxel, ascending.  *K receives the
// number of occupied voxels; reps must hold n entries.
int hor_select(const float* pts, int64_t n, float s, const float aspect[3],
               int32_t* reps, int64_t* K) {
    if (!pts || !reps || !K || n <= 0) return OR_ERR_INVALID;
    Ctx c;
    int st = bounding_box(pts, n, aspect, &c);
    if (st != OR_OK) return st;
    float v[3];
    int64_t fmin[3];
    if (!voxel_size(c, s, v) || !min_cells(c, v, fmin)) return OR_ERR_RANGE;
    std::unordered_map<uint64_t, uint64_t> table;
    for (int64_t i = 0; i < n; ++i) {
        uint64_t key;
        float f[3];
        if (!voxel_key(pts + 3 * i, v, fmin, &key, f)) return OR_ERR_RANGE;
        float d2 = centre_dist2(pts + 3 * i, v, f);
        uint64_t packed = (static_cast<uint64_t>(float_bits(d2)) << 32) |
                          static_cast<uint32_t>(i);
        auto it = table.find(key);
        if (it == table.end()) table.emplace(key, packed);
        else if (packed < it->second) it->second = packed;
    }
    std::vector<int32_t> r;
    for (const auto& kv : table) r.push_back(static_cast<int32_t>(kv.second & 0xffffffffu));
    std::sort(r.begin(), r.end());
    std::copy(r.begin(), r.end(), reps);
    *K = static_cast<int64_t>(r.size());
    return OR_OK;
}

uint64_t hor_priority(uint64_t key) { return splitmix_finalise(key); }

uint64_t hor_random(uint32_t seed, uint64_t counter) { return random_draw(seed, counter); }

// Representative coordinates of a one-layer call (Table 6 point-selection
// strategies).  out_idx receives the m ascending indices hor_sample gives;
// out_xyz (3m floats) the coordinates that stand for each: for an index that
// represents its voxel at s* (the voxel's centre-closest point, or its random
// draw for RA), the point itself (CC, RA), the voxel centre v * (g + 0.5) in
// binary32 (CE), or the voxel mean (ME); for an index added by the shortfall
// fill, the point itself.
//
// The mean is computed in fixed point so that it does not depend on the
// order of summation: with M the largest |coordinate| of the cloud and
// 2^(k-1) <= M < 2^k (k = 0 when M = 0), every coordinate x is taken as the
// integer X = round-half-even(x * 2^(30 - k)); a voxel's mean on one axis is
// RN32(RN64(RN64(sum X) / count) * 2^(k - 30)).
int hor_sample_xyz(const float* pts, int64_t n, int64_t m, const hor_params* p,
                   int32_t* out_idx, float* out_xyz, hor_layer_trace* tr) {
    int st = check_params(p);
    if (st != OR_OK) return st;
    if (p->layers != 1) return OR_ERR_INVALID;
    hor_layer_trace rec;
    std::memset(&rec, 0, sizeof rec);
    st = hor_sample(pts, n, m, p, out_idx, &rec);
    if (st != OR_OK || m == 0) {
        if (tr) *tr = rec;
        return st;
    }
    if (tr) *tr = rec;
    for (int64_t r = 0; r < m; ++r)
        for (int a = 0; a < 3; ++a) out_xyz[3 * r + a] = pts[3 * int64_t(out_idx[r]) + a];
    if (p->select == OR_SEL_CC || p->select == OR_SEL_RA) return OR_OK;

    Ctx c;
    st = bounding_box(pts, n, p->aspect, &c);
    if (st != OR_OK) return st;
    float v[3];
    int64_t fmin[3];
    if (!voxel_size(c, rec.s_star, v) || !min_cells(c, v, fmin)) return OR_ERR_RANGE;
    // the centre-closest point of every voxel, and the fixed-point sums
    float M = 0.0f;
    for (int64_t i = 0; i < 3 * n; ++i) M = std::max(M, std::fabs(pts[i]));
    int k = 0;
    if (M > 0.0f) std::frexp(M, &k);  // M = f * 2^k, f in [0.5, 1)
    const int q = 30 - k;
    struct Acc { uint64_t best; int64_t sum[3]; int64_t count; float f[3]; };
    std::unordered_map<uint64_t, Acc> vox;
    for (int64_t i = 0; i < n; ++i) {
        uint64_t key;
        float f[3];
        if (!voxel_key(pts + 3 * i, v, fmin, &key, f)) return OR_ERR_RANGE;
        uint64_t packed = (static_cast<uint64_t>(float_bits(centre_dist2(pts + 3 * i, v, f))) << 32) |
                          static_cast<uint32_t>(i);
        auto it = vox.find(key);
        if (it == vox.end()) {
            Acc acc;
            acc.best = packed;
            acc.count = 0;
            for (int a = 0; a < 3; ++a) { acc.sum[a] = 0; acc.f[a] = f[a]; }
            it = vox.emplace(key, acc).first;
        }
        Acc& acc = it->second;
        if (packed < acc.best) acc.best = packed;
        for (int a = 0; a < 3; ++a)
            acc.sum[a] += std::llrint(std::ldexp(static_cast<double>(pts[3 * i + a]), q));
        acc.count += 1;
    }
    for (int64_t r = 0; r < m; ++r) {
        const int32_t i = out_idx[r];
        uint64_t key;
        float f[3];
        voxel_key(pts + 3 * int64_t(i), v, fmin, &key, f);
        const Acc& acc = vox.at(key);
        if (static_cast<int32_t>(acc.best & 0xffffffffu) != i) continue;  // shortfall fill
        for (int a = 0; a < 3; ++a) {
            if (p->select == OR_SEL_CE) {
                const float cen = acc.f[a] + 0.5f;
                out_xyz[3 * r + a] = v[a] * cen;
            } else {
                const double mean = static_cast<double>(acc.sum[a]) / static_cast<double>(acc.count);
                out_xyz[3 * r + a] = static_cast<float>(std::ldexp(mean, -q));
            }
        }
    }
    return OR_OK;
}

float hor_s_hi(const float* pts, int64_t n, const float aspect[3]) {
    Ctx c;
    if (bounding_box(pts, n, aspect, &c) != OR_OK) return -1.0f;
    return c.s_hi;
}

// Point spacing of a sampled subset (the distributions of Fig. 3, Section
// 3.1): for each subset point, the smallest squared distance to any other
// subset point, binary32 (dx*dx + dy*dy) + dz*dz without fusion; +inf for a
// subset of one point.  Brute force over all pairs.
int hor_spacing(const float* pts, int64_t n, const int32_t* idx, int64_t m, float* out_d2) {
    if (!pts || !idx || !out_d2 || m < 0 || n < 0) return OR_ERR_INVALID;
    for (int64_t r = 0; r < m; ++r)
        if (idx[r] < 0 || idx[r] >= n) return OR_ERR_INVALID;
    for (int64_t r = 0; r < m; ++r) {
        const float* a = pts + 3 * int64_t(idx[r]);
        float best = INFINITY;
        for (int64_t q = 0; q < m; ++q) {
            if (q == r) continue;
            const float* b = pts + 3 * int64_t(idx[q]);
            float dx = a[0] - b[0], dy = a[1] - b[1], dz = a[2] - b[2];
            float xx = dx * dx, yy = dy * dy, zz = dz * dz;
            float d2 = (xx + yy) + zz;
            if (d2 < best) best = d2;
        }
        out_d2[r] = best;
    }
    return OR_OK;
}

// Grouping around sampled centres, the step that follows sampling in the
// sample-group-aggregate block (Section 3.1; the ball query of PointNet++):
// for centre j (the point centres[j]), the nsample smallest indices k with
// (dx*dx + dy*dy) + dz*dz < radius*radius in binary32, ascending; if fewer
// qualify, the remaining slots repeat the smallest.  The centre itself always
// qualifies.  out_xyz (optional) receives p_k - c_j per slot.
int hor_ball_query(const float* pts, int64_t n, const int32_t* centres, int64_t m, float radius,
                   int32_t nsample, int32_t* out_idx, float* out_xyz) {
    if (!pts || (m > 0 && (!centres || !out_idx)) || n < 0 || m < 0 || nsample < 1) return OR_ERR_INVALID;
    if (!(radius > 0.0f) || !std::isfinite(radius)) return OR_ERR_INVALID;
    const float r2 = radius * radius;
    for (int64_t j = 0; j < m; ++j) {
        if (centres[j] < 0 || centres[j] >= n) return OR_ERR_INVALID;
        const float* c = pts + 3 * int64_t(centres[j]);
        int32_t cnt = 0;
        int32_t* row = out_idx + j * int64_t(nsample);
        for (int64_t k = 0; k < n && cnt < nsample; ++k) {
            const float* q = pts + 3 * k;
            float dx = q[0] - c[0], dy = q[1] - c[1], dz = q[2] - c[2];
            float xx = dx * dx, yy = dy * dy, zz = dz * dz;
            float d2 = (xx + yy) + zz;
            if (d2 < r2) row[cnt++] = static_cast<int32_t>(k);
        }
        for (int32_t s = cnt; s < nsample; ++s) row[s] = row[0];
        if (out_xyz)
            for (int32_t s = 0; s < nsample; ++s)
                for (int a = 0; a < 3; ++a)
                    out_xyz[(j * int64_t(nsample) + s) * 3 + a] = pts[3 * int64_t(row[s]) + a] - c[a];
    }
    return OR_OK;
}

// Farthest point sampling (Eq. 1), the paper's comparator: start at index 0,
// squared distances in binary32 without fusion, argmax ties to the lowest
// index, selected points never chosen again.
int hor_fps(const float* pts, int64_t n, int64_t m, int32_t* out) {
    if (n < 0 || m < 0 || m > n || n >= (int64_t(1) << 31)) return OR_ERR_INVALID;
    if (m == 0) return OR_OK;
    std::vector<float> best(static_cast<size_t>(n), INFINITY);
    std::vector<uint8_t> chosen(static_cast<size_t>(n), 0);
    int64_t last = 0;
    out[0] = 0;
    chosen[0] = 1;
    for (int64_t j = 1; j < m; ++j) {
        const float* q = pts + 3 * last;
        int64_t arg = -1;
        float bestd = -1.0f;
        for (int64_t i = 0; i < n; ++i) {
            if (chosen[i]) continue;
            const float* pi = pts + 3 * i;
            float dx = pi[0] - q[0], dy = pi[1] - q[1], dz = pi[2] - q[2];
            float xx = dx * dx, yy = dy * dy, zz = dz * dz;
            float d2 = (xx + yy) + zz;
            if (d2 < best[i]) best[i] = d2;
            if (best[i] > bestd) { bestd = best[i]; arg = i; }
        }
        out[j] = static_cast<int32_t>(arg);
        chosen[arg] = 1;
        last = arg;
    }
    return OR_OK;
}

}  // extern "C"
