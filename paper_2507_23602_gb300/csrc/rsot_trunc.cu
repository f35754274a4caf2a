// Truncated dual + gradient evaluation (Algorithm 2 with I_q = {j : c(x_q,y_j) < C}).
//
// Spatial index (replaces the paper's R-tree, Sec. 4.1): a uniform grid of
// 2^b cells per axis over the bounding box of points and targets.  Points and
// targets are ordered by the Morton (Z-order) index of their cell, ties by
// their input index (a deterministic bitonic sort on the GPU, built once per
// problem).  Consecutive runs of the sorted order form tiles -- 1024 points or
// 256 targets -- that are spatially compact; each tile carries its bounding
// box.  Per evaluation, a (point tile, target tile) pair is a candidate when
// the boxes are closer than the largest cutoff radius of their members; every
// candidate pair of points and targets is then tested (c < C_qj, strict)
// inside the kernels, so the sums run over I_q as in Algorithm 2.
//
// Work is a queue of items (point tile, chunk of candidate target tiles) for
// pass 1 and (target tile, chunk of candidate point tiles) for pass 2,
// consumed by persistent CTAs through an atomic counter.  Partial results are
// stored per item and merged in a fixed order, so results do not depend on
// which CTA ran which item.
//
// The cutoff is per pair, c(x_q, y_j) < alpha_q + beta_j (rsot_cutoff.cu:
// alpha_q = C, beta_j = 0 for a radius; the separable psi-aware cutoff
// otherwise).  Mixed precision uses the log2-domain quantities of the dense
// path (rsot_dense.cu): r_qj = c_j + x'_q.w_j, and with c = |x'_q - y'_j|^2 / 2
//   k |x'_q - y'_j|^2 < 2k (alpha_q + beta_j)
//     <=>   r_qj - (b_j - 2k beta_j) > k |x'_q|^2 - 2k alpha_q  (=: A_q),
// b_j - 2k beta_j being the per-target test constant.  Blocks and tiles carry
// the ranges of alpha and beta over their members for the culling.  The FP64
// truncated evaluation reuses the dense FP64 kernels with the predicate
// (rsot_dense.cu).
#include <math.h>
#include <stdio.h>

#include <algorithm>

#include "rsot_internal.cuh"
#include "rsot_tc.cuh"

namespace rsot {

struct __align__(16) Rec12 {
    float4 a, b, c;
};

struct Grid {
    int b = 0, G = 0;
    double lo[3] = {0, 0, 0};
    double h = 0.0;
    int64_t nqt = 0, nt = 0;             // padded sorted counts
    int ptiles = 0, ttiles = 0, tw = 0, pw = 0;
    int ch1 = 0, ch2 = 0;
    int64_t items1_max = 0, items2_max = 0;
    int slots1 = 0, slots2 = 0;
    int *perm_q = nullptr, *perm_t = nullptr;
    float *xs = nullptr;                  // [d][nqt]
    double *x64 = nullptr, *mass = nullptr, *lm2 = nullptr;
    double *y64 = nullptr, *nu = nullptr, *lnu = nullptr;
    float *pbox = nullptr, *tbox = nullptr;
    uint32_t *bits_pt = nullptr, *bits_tp = nullptr;
    int *cnt1 = nullptr, *cnt2 = nullptr, *off1 = nullptr, *off2 = nullptr, *counters = nullptr;
    float *Aq = nullptr;
    Rec12 *tdup = nullptr, *ppair = nullptr;
    float2 *part1 = nullptr;
    double *part2 = nullptr;
    double *lse_s = nullptr;
    double *blockJ = nullptr;
    int nblk_comb = 0;
    // tensor-core passes: block balls (centre, radius; radius < 0: no member),
    // operand records in sorted order, per-target b_j, per-point shifts u_q
    float4 *pball64 = nullptr, *pball8 = nullptr, *tball64 = nullptr, *tball8 = nullptr;
    Rec16 *prec_s = nullptr, *trec_s = nullptr;
    float *b_s = nullptr, *u_s = nullptr;
    // per evaluation: (min, max) of alpha over point blocks of 16 / 8 and of
    // beta over target blocks of 8 / 16, maxima over point / target tiles
    float2 *pal64 = nullptr, *pal8 = nullptr, *tbe8 = nullptr, *tbe64 = nullptr;
    float *ptmax = nullptr, *ttmax = nullptr;
    // initial pass-1 shift per point: ceil of the exponent of its nearest target
    // (psi-aware cutoffs: a kept term, a lower bound of the maximum), -inf else
    float *m0_s = nullptr;
    // block-skip tensor-core passes: boxes of 512-point / 512- and 1024-target
    // runs (once), maxima of alpha / beta over them (per evaluation), partials
    // in the item layout (tile * chunks + chunk) and its offsets
    float *pbox512 = nullptr, *tbox512 = nullptr, *tbox1024 = nullptr;
    float *pa512 = nullptr, *tb512 = nullptr, *tb1024 = nullptr;
    float2 *part1b = nullptr;
    double *part2b = nullptr;
    Rec8 *pdup_s = nullptr;   // FP32 block-skip pass 2: sorted point records (per evaluation)
    float *nAq_s = nullptr;   // FP32 block-skip pass 2: -A_q 2^64 of the sorted points (per evaluation)
    int *off1b = nullptr, *off2b = nullptr;
    int k1b = 0, k2b = 0;
};

namespace {

constexpr int PT = 1024;          // points per tile
constexpr int TT = 256;           // targets per tile
constexpr int L_THREADS = 128;    // pass-1 CTA (8 points / thread)
constexpr int L_PP = 4;
constexpr int L_SUB = 8;          // targets per max sub-tile
constexpr float L_THR = 32.0f;
constexpr int G_THREADS = 64;     // pass-2 CTA (4 targets / thread)
constexpr int G_TPT = 4;
constexpr int G_STAGE = 256;      // point-pair records per pass-2 stage (512 points)
constexpr int MAX_CH = 64;

inline int64_t round_up(int64_t a, int64_t b) { return (a + b - 1) / b * b; }

// ---------------------------------------------------------------- grid build
__device__ __forceinline__ unsigned spread3(unsigned v) {   // 10 bits -> every 3rd bit
    v &= 0x3ffu;
    v = (v | (v << 16)) & 0x030000FFu;
    v = (v | (v << 8)) & 0x0300F00Fu;
    v = (v | (v << 4)) & 0x030C30C3u;
    v = (v | (v << 2)) & 0x09249249u;
    return v;
}
__device__ __forceinline__ unsigned spread2(unsigned v) {   // 15 bits -> every 2nd bit
    v &= 0x7fffu;
    v = (v | (v << 8)) & 0x00FF00FFu;
    v = (v | (v << 4)) & 0x0F0F0F0Fu;
    v = (v | (v << 2)) & 0x33333333u;
    v = (v | (v << 1)) & 0x55555555u;
    return v;
}

__global__ void k_morton_keys(const double *__restrict__ c64, int64_t cnt, int64_t npow2, int d,
                              double lo0, double lo1, double lo2, double inv_h, int G,
                              unsigned long long *__restrict__ keys) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= npow2) return;
    if (i >= cnt) {
        keys[i] = ~0ull;
        return;
    }
    const double lo[3] = {lo0, lo1, lo2};
    unsigned cell[3] = {0, 0, 0};
    for (int k = 0; k < d; ++k) {
        double t = (c64[i * d + k] - lo[k]) * inv_h;
        int ci = (int)floor(t);
        ci = ci < 0 ? 0 : (ci >= G ? G - 1 : ci);
        cell[k] = (unsigned)ci;
    }
    const unsigned code = (d == 3) ? (spread3(cell[0]) | (spread3(cell[1]) << 1) | (spread3(cell[2]) << 2))
                                   : (spread2(cell[0]) | (spread2(cell[1]) << 1));
    keys[i] = ((unsigned long long)code << 32) | (unsigned long long)i;
}

__global__ void k_bitonic_step(unsigned long long *__restrict__ a, int64_t n, int64_t j, int64_t k) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int64_t ixj = i ^ j;
    if (ixj > i) {
        const bool up = (i & k) == 0;
        const unsigned long long x = a[i], y = a[ixj];
        if ((x > y) == up) {
            a[i] = y;
            a[ixj] = x;
        }
    }
}

// sorted position s -> original index; gather FP32/FP64 copies in sorted order
__global__ void k_gather_points(const unsigned long long *__restrict__ keys, int64_t nq, int64_t nqt,
                                int d, const double *__restrict__ x64, const double *__restrict__ mass,
                                const double *__restrict__ lm2, int *__restrict__ perm, float *__restrict__ xs,
                                double *__restrict__ x64s, double *__restrict__ mass_s,
                                double *__restrict__ lm2_s) {
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nqt) return;
    if (s < nq) {
        const int64_t o = (int64_t)(keys[s] & 0xffffffffull);
        perm[s] = (int)o;
        for (int k = 0; k < d; ++k) {
            const double v = x64[o * d + k];
            x64s[s * d + k] = v;
            xs[k * nqt + s] = (float)v;
        }
        mass_s[s] = mass[o];
        lm2_s[s] = lm2[o];
    } else {
        perm[s] = -1;
        for (int k = 0; k < d; ++k) {
            x64s[s * d + k] = 0.0;
            xs[k * nqt + s] = 0.0f;
        }
        mass_s[s] = 0.0;
        lm2_s[s] = -INFINITY;
    }
}

__global__ void k_gather_targets(const unsigned long long *__restrict__ keys, int64_t n, int64_t nt,
                                 int d, const double *__restrict__ y64, const double *__restrict__ nu,
                                 const double *__restrict__ lnu, int *__restrict__ perm,
                                 double *__restrict__ y64s, double *__restrict__ nu_s,
                                 double *__restrict__ lnu_s) {
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nt) return;
    if (s < n) {
        const int64_t o = (int64_t)(keys[s] & 0xffffffffull);
        perm[s] = (int)o;
        for (int k = 0; k < d; ++k) y64s[s * d + k] = y64[o * d + k];
        nu_s[s] = nu[o];
        lnu_s[s] = lnu[o];
    } else {
        perm[s] = -1;
        for (int k = 0; k < d; ++k) y64s[s * d + k] = 0.0;
        nu_s[s] = 0.0;
        lnu_s[s] = -INFINITY;
    }
}

// bounding box of each tile over its real members (FP32 coordinates)
__global__ void k_tile_boxes(const double *__restrict__ c64s, int64_t cnt, int d, int tile,
                             int ntiles, float *__restrict__ box) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ntiles) return;
    float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    const int64_t a = (int64_t)t * tile, e = min((int64_t)(t + 1) * tile, cnt);
    for (int64_t s = a; s < e; ++s)
        for (int k = 0; k < d; ++k) {
            const float v = (float)c64s[s * d + k];
            lo[k] = fminf(lo[k], v);
            hi[k] = fmaxf(hi[k], v);
        }
    for (int k = 0; k < 3; ++k) {
        if (k >= d) {
            lo[k] = 0.f;
            hi[k] = 0.f;
        }
        box[t * 6 + k] = lo[k];
        box[t * 6 + 3 + k] = hi[k];
    }
}


// Bounding ball (centre, radius; radius -1 for a block without members) of
// each run of B consecutive sorted members, from the FP64 copies (translated
// coordinates, [cnt_pad][d]).  The radius is the half diagonal of the block's
// box, rounded up by 1e-6 relative.
__global__ void k_block_balls(const double *__restrict__ c64s, int64_t cnt, int d, int B,
                              int64_t nblocks, float4 *__restrict__ ball) {
    const int64_t bi = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (bi >= nblocks) return;
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    const int64_t a = bi * B, e = min((bi + 1) * B, cnt);
    for (int64_t q = a; q < e; ++q)
        for (int k = 0; k < d; ++k) {
            lo[k] = fmin(lo[k], c64s[q * d + k]);
            hi[k] = fmax(hi[k], c64s[q * d + k]);
        }
    if (a >= e) {
        ball[bi] = make_float4(0.f, 0.f, 0.f, -1.f);
        return;
    }
    double c[3] = {0.0, 0.0, 0.0}, r2 = 0.0;
    for (int k = 0; k < d; ++k) {
        c[k] = 0.5 * (lo[k] + hi[k]);
        r2 += 0.25 * (hi[k] - lo[k]) * (hi[k] - lo[k]);
    }
    ball[bi] = make_float4((float)c[0], (float)c[1], (float)c[2], (float)(sqrt(r2) * (1.0 + 1e-6) + 1e-9));
}

// tensor-core point records of the sorted points (X = P x', rsot_tc.cuh)
__global__ void k_point_recs_s(const float *__restrict__ xs, int64_t nqt, int d, float P,
                               Rec16 *__restrict__ prec) {
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nqt) return;
    float X[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) X[k] = k < d ? xs[k * nqt + q] * P : 0.0f;
    prec[q] = make_point_rec(X, 0.0f);
}

// ------------------------------------------------------------- per evaluation
// A_q = k |x'_q|^2 - 2k alpha_q (FP32, computed once so that both passes agree).
// With anchored (psi-aware) cutoffs alpha_q = c_qn - psi_n - eps ln nu_n, the
// exponent of the anchor pair is r_qn = b_n + k|x'_q|^2 - 2k c_qn = A_q - 2k psi_c:
// M0 = ceil(r_qn) starts the pass-1 running maximum there.
__global__ void k_trunc_A(const float *__restrict__ xs, int64_t nq, int64_t nqt, int d, float k,
                          const double *__restrict__ alpha, const int *__restrict__ perm_q,
                          double k2, const double *__restrict__ psi, int anchored,
                          float *__restrict__ Aq, float *__restrict__ M0) {
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nqt) return;
    if (s >= nq) {
        Aq[s] = INFINITY;
        M0[s] = -INFINITY;
        return;
    }
    float r2 = 0.f;
    for (int t = 0; t < d; ++t) {
        const float v = xs[t * nqt + s];
        r2 = fmaf(v, v, r2);
    }
    const double a = alpha[perm_q[s]];
    Aq[s] = fmaf(k, r2, -(float)(k2 * a));
    M0[s] = anchored ? ceilf(fmaf(k, r2, -(float)(k2 * (a + psi[0])))) : -INFINITY;
}

// (min, max) of v[perm[s]] over runs of 8 sorted members (real members only:
// (+inf, -inf) for a block without any)
__global__ void k_ranges8(const double *__restrict__ v, const int *__restrict__ perm, int64_t cnt,
                          int64_t nblocks, float2 *__restrict__ out) {
    const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nblocks) return;
    double lo = INFINITY, hi = -INFINITY;
    for (int64_t s = b * 8; s < min((b + 1) * 8, cnt); ++s) {
        const double a = v[perm[s]];
        lo = fmin(lo, a);
        hi = fmax(hi, a);
    }
    // rounded outwards to FP32
    float flo = (float)lo, fhi = (float)hi;
    if ((double)flo > lo) flo = nextafterf(flo, -INFINITY);
    if ((double)fhi < hi) fhi = nextafterf(fhi, INFINITY);
    out[b] = make_float2(flo, fhi);
}

// merge runs of f consecutive ranges; optionally only the maxima
__global__ void k_ranges_merge(const float2 *__restrict__ in, int64_t nin, int f,
                               float2 *__restrict__ out, float *__restrict__ out_max, int64_t nout) {
    const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nout) return;
    float lo = INFINITY, hi = -INFINITY;
    for (int64_t i = b * f; i < min((b + 1) * f, nin); ++i) {
        lo = fminf(lo, in[i].x);
        hi = fmaxf(hi, in[i].y);
    }
    if (out) out[b] = make_float2(lo, hi);
    if (out_max) out_max[b] = hi;
}

__device__ __forceinline__ float box_dist2(const float *a, const float *b) {
    float s = 0.f;
    for (int k = 0; k < 3; ++k) {
        const float g = fmaxf(0.f, fmaxf(a[k] - b[3 + k], b[k] - a[3 + k]));
        s = fmaf(g, g, s);
    }
    return s;
}

// candidate (point tile, target tile) pairs: bit matrices in both orientations
// a pair is a candidate when its boxes are closer than the largest cutoff radius
// of its members, sqrt(2 (max alpha + max beta)), widened by 1e-5 relative
__global__ void k_tile_pairs(const float *__restrict__ pbox, const float *__restrict__ tbox,
                             int ptiles, int ttiles, int tw, int pw, const float *__restrict__ ptmax,
                             const float *__restrict__ ttmax,
                             uint32_t *__restrict__ bits_pt, uint32_t *__restrict__ bits_tp,
                             int *__restrict__ cnt1, int *__restrict__ cnt2) {
    __shared__ int s_cnt;
    const int p = blockIdx.x;
    if (threadIdx.x == 0) s_cnt = 0;
    __syncthreads();
    float pb[6];
    for (int k = 0; k < 6; ++k) pb[k] = pbox[p * 6 + k];
    const bool pempty = !(pb[0] <= pb[3]);
    const float pa = ptmax[p];
    int mine = 0;
    for (int t0 = 0; t0 < tw * 32; t0 += blockDim.x) {
        const int t = t0 + threadIdx.x;
        bool cand = false;
        if (t < ttiles && !pempty) {
            float tb[6];
            for (int k = 0; k < 6; ++k) tb[k] = tbox[t * 6 + k];
            const float rr = sqrtf(fmaxf(0.f, 2.f * (pa + ttmax[t]))) * (1.0f + 1e-5f) + 1e-6f;
            cand = (tb[0] <= tb[3]) && box_dist2(pb, tb) < rr * rr;
        }
        const unsigned bal = __ballot_sync(0xffffffffu, cand);
        if ((threadIdx.x & 31) == 0 && t < tw * 32) bits_pt[(size_t)p * tw + t / 32] = bal;
        if (cand) {
            atomicOr(&bits_tp[(size_t)t * pw + p / 32], 1u << (p & 31));
            atomicAdd(&cnt2[t], 1);
            ++mine;
        }
    }
    atomicAdd(&s_cnt, mine);
    __syncthreads();
    if (threadIdx.x == 0) cnt1[p] = s_cnt;
}

// item offsets: off[i] = sum_{i' < i} ceil(cnt[i'] / ch); one block
__global__ void k_item_offsets(const int *__restrict__ cnt1, int ptiles, int ch1,
                               const int *__restrict__ cnt2, int ttiles, int ch2,
                               int *__restrict__ off1, int *__restrict__ off2,
                               int *__restrict__ counters) {
    if (threadIdx.x == 0) {
        int s = 0;
        for (int i = 0; i < ptiles; ++i) {
            off1[i] = s;
            s += (cnt1[i] + ch1 - 1) / ch1;
        }
        off1[ptiles] = s;
        counters[0] = 0;
    } else if (threadIdx.x == 32) {
        int s = 0;
        for (int i = 0; i < ttiles; ++i) {
            off2[i] = s;
            s += (cnt2[i] + ch2 - 1) / ch2;
        }
        off2[ttiles] = s;
        counters[1] = 0;
    }
}

// target records in sorted order: (w0,w0,w1,w1) (w2,w2,c,c) (-b,-b,0,0)
__global__ void k_prep_trunc(const double *__restrict__ psi, const int *__restrict__ perm_t,
                             const double *__restrict__ y64s, const double *__restrict__ lnu_s,
                             int64_t n, int64_t nt, int d, double eps, Rec12 *__restrict__ tdup,
                             double *__restrict__ psinu_part, const double *__restrict__ nu_s,
                             int *__restrict__ flags, Rec16 *__restrict__ trec, float *__restrict__ bs,
                             double inv_P, int *__restrict__ gate, const double *__restrict__ beta) {
    __shared__ double sh[32];
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const double psic = psi[0];
    const double k = kLog2e / (2.0 * eps);
    double contrib = 0.0;
    if (s < nt) {
        float w[3] = {0.f, 0.f, 0.f};
        float c = kPadC, nb = kPadC;
        if (s < n) {
            const double ps = psi[perm_t[s]];
            if (!isfinite(ps)) atomicOr(flags, kErrNonfinitePsi);
            const double b = ((ps - psic) / eps + lnu_s[s]) * kLog2e;
            double yy = 0.0;
            for (int t = 0; t < d; ++t) {
                const double yt = y64s[s * d + t];
                w[t] = (float)(2.0 * k * yt);
                yy += yt * yt;
            }
            c = (float)(b - k * yy);
            // test constant b_j - 2k beta_j (cutoff c < alpha_q + beta_j)
            nb = (float)(2.0 * k * beta[perm_t[s]] - b);
            contrib = ps * nu_s[s];
        }
        Rec12 r;
        r.a = make_float4(w[0], w[0], w[1], w[1]);
        r.b = make_float4(w[2], w[2], c, c);
        r.c = make_float4(nb, nb, 0.f, 0.f);
        tdup[s] = r;
        if (trec) {
            // tensor-core operands (rsot_tc.cuh) and b_j (+inf for padding: the
            // truncation test r - b_j > A_q then fails)
            float W[3] = {0.f, 0.f, 0.f};
            float C = -256.0f * TC_RANGE;
            bool ok = true;
            if (s < n) {
                for (int t = 0; t < d; ++t) {
                    W[t] = (float)(2.0 * k * y64s[s * d + t] * inv_P);
                    ok = ok && fabsf(W[t]) < TC_RANGE;
                }
                C = fmaxf(c, -256.0f * TC_RANGE);
                ok = ok && C < 256.0f * TC_RANGE;
            }
            if (!ok) atomicOr(gate, 1);
            trec[s] = make_target_rec(W, C);
            bs[s] = s < n ? -nb : INFINITY;
        }
    }
    const double v = block_sum_d(contrib, sh);
    if (threadIdx.x == 0) psinu_part[blockIdx.x] = v;
}

// k-th chunk of set bits of a bit row -> list (thread 0 only)
__device__ int collect_bits(const uint32_t *__restrict__ row, int words, int skip, int ch, int *list) {
    int got = 0;
    for (int w = 0; w < words && got < ch; ++w) {
        uint32_t bits = row[w];
        const int pc = __popc(bits);
        if (skip >= pc) {
            skip -= pc;
            continue;
        }
        while (bits && got < ch) {
            const int b = __ffs(bits) - 1;
            bits &= bits - 1;
            if (skip > 0) {
                --skip;
                continue;
            }
            list[got++] = w * 32 + b;
        }
    }
    return got;
}

__device__ __forceinline__ int find_row(const int *__restrict__ off, int rows, int item) {
    int lo = 0, hi = rows;   // off[lo] <= item < off[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (off[mid] <= item) lo = mid;
        else hi = mid;
    }
    return lo;
}

// ------------------------------------------------------------------- pass 1
template <int D>
__global__ void __launch_bounds__(L_THREADS, 3)
    k_lse_trunc(const float *__restrict__ xs, int64_t nqt, const float *__restrict__ Aq,
                const Rec12 *__restrict__ tdup, const uint32_t *__restrict__ bits_pt, int tw,
                const int *__restrict__ off1, int ptiles, int ch1, int *__restrict__ counter,
                float2 *__restrict__ part1, unsigned long long *__restrict__ pairs,
                int *__restrict__ flags, const int *__restrict__ gate = nullptr) {
    // as the fallback of the tensor-core pass, run only when the gate asks for it
    if (gate && !(*gate & 1)) return;
    __shared__ __align__(128) Rec12 sm[2][TT];
    __shared__ __align__(8) uint64_t full[2];
    __shared__ int s_item, s_p, s_cnt, s_abort[2];
    __shared__ int s_list[MAX_CH];
    __shared__ unsigned long long s_pairs;
    const int tid = threadIdx.x;
    if (tid == 0) {
        for (int s = 0; s < 2; ++s) mbar_init(&full[s], 1);
        fence_barrier_init();
        s_abort[0] = s_abort[1] = 0;
        s_pairs = 0;
    }
    __syncthreads();
    const int total = off1[ptiles];
    unsigned git = 0;
    unsigned long long mycnt = 0;
    bool aborted = false;
    for (;;) {
        if (tid == 0) {
            const int it = atomicAdd(counter, 1);
            s_item = it;
            if (it < total) {
                const int p = find_row(off1, ptiles, it);
                s_p = p;
                s_cnt = collect_bits(bits_pt + (size_t)p * tw, tw, (it - off1[p]) * ch1, ch1, s_list);
            }
        }
        __syncthreads();
        const int item = s_item;
        if (item >= total) break;
        const int p = s_p, cnt = s_cnt;
        if (tid == 0) {
            for (int s = 0; s < 2 && s < cnt; ++s) {
                const unsigned slot = (git + s) & 1u;
                mbar_expect_tx(&full[slot], TT * sizeof(Rec12));
                bulk_g2s(sm[slot], tdup + (int64_t)s_list[s] * TT, TT * sizeof(Rec12), &full[slot]);
            }
        }
        const int64_t q0 = (int64_t)p * PT;
        float2 X[L_PP][3], A[L_PP];
#pragma unroll
        for (int pp = 0; pp < L_PP; ++pp) {
            const int64_t q = q0 + 2 * (pp * L_THREADS + tid);
#pragma unroll
            for (int k = 0; k < 3; ++k)
                X[pp][k] = (k < D) ? *reinterpret_cast<const float2 *>(xs + k * nqt + q)
                                   : make_float2(0.f, 0.f);
            A[pp] = *reinterpret_cast<const float2 *>(Aq + q);
        }
        float2 M[L_PP], Sf[L_PP];
        double2 Sd[L_PP];
#pragma unroll
        for (int pp = 0; pp < L_PP; ++pp) {
            M[pp] = make_float2(kPadC, kPadC);
            Sf[pp] = make_float2(0.f, 0.f);
            Sd[pp] = make_double2(0.0, 0.0);
        }
        unsigned icnt = 0;
        for (int it = 0; it < cnt; ++it) {
            const unsigned gs = git + it, slot = gs & 1u, ph = (gs >> 1) & 1u;
            if (!mbar_wait(&full[slot], ph)) {
                s_abort[it & 1] = 1;
                atomicOr(flags, kErrTimeout);
            } else {
                const Rec12 *T = sm[slot];
#pragma unroll 1
                for (int t0 = 0; t0 < TT; t0 += L_SUB) {
                    float2 r[L_PP][L_SUB];
#pragma unroll
                    for (int t = 0; t < L_SUB; ++t) {
                        const float4 a = T[t0 + t].a, b = T[t0 + t].b, e = T[t0 + t].c;
                        const float2 w0 = make_float2(a.x, a.y), w1 = make_float2(a.z, a.w);
                        const float2 w2 = make_float2(b.x, b.y), c = make_float2(b.z, b.w);
                        const float2 nb = make_float2(e.x, e.y);
#pragma unroll
                        for (int pp = 0; pp < L_PP; ++pp) {
                            float2 acc = c;
                            if (D == 3) acc = __ffma2_rn(X[pp][2], w2, acc);
                            acc = __ffma2_rn(X[pp][1], w1, acc);
                            acc = __ffma2_rn(X[pp][0], w0, acc);
                            const float2 v = __fadd2_rn(acc, nb);
                            const bool px = v.x > A[pp].x, py = v.y > A[pp].y;
                            icnt += (unsigned)px + (unsigned)py;
                            r[pp][t] = make_float2(px ? acc.x : -INFINITY, py ? acc.y : -INFINITY);
                        }
                    }
#pragma unroll
                    for (int pp = 0; pp < L_PP; ++pp) {
                        float mx = r[pp][0].x, my = r[pp][0].y;
#pragma unroll
                        for (int t = 1; t + 1 < L_SUB; t += 2) {
                            mx = max3f(mx, r[pp][t].x, r[pp][t + 1].x);
                            my = max3f(my, r[pp][t].y, r[pp][t + 1].y);
                        }
                        mx = fmaxf(mx, r[pp][L_SUB - 1].x);
                        my = fmaxf(my, r[pp][L_SUB - 1].y);
                        if (mx > M[pp].x + L_THR) {
                            const float mn = ceilf(mx), dl = M[pp].x - mn;
                            Sf[pp].x *= pow2_int_f(dl);
                            Sd[pp].x *= pow2_int_d(dl);
                            M[pp].x = mn;
                        }
                        if (my > M[pp].y + L_THR) {
                            const float mn = ceilf(my), dl = M[pp].y - mn;
                            Sf[pp].y *= pow2_int_f(dl);
                            Sd[pp].y *= pow2_int_d(dl);
                            M[pp].y = mn;
                        }
                        const float2 nm = make_float2(-M[pp].x, -M[pp].y);
                        float2 acc = make_float2(0.f, 0.f);
#pragma unroll
                        for (int t = 0; t < L_SUB; ++t) {
                            const float2 e = __fadd2_rn(r[pp][t], nm);
                            acc = __fadd2_rn(acc, make_float2(ex2_approx(e.x), ex2_approx(e.y)));
                        }
                        Sf[pp] = __fadd2_rn(Sf[pp], acc);
                    }
                }
            }
            __syncthreads();
            aborted = s_abort[it & 1] != 0;
            if (aborted) break;
            if (tid == 0 && it + 2 < cnt) {
                mbar_expect_tx(&full[slot], TT * sizeof(Rec12));
                bulk_g2s(sm[slot], tdup + (int64_t)s_list[it + 2] * TT, TT * sizeof(Rec12), &full[slot]);
            }
#pragma unroll
            for (int pp = 0; pp < L_PP; ++pp) {
                Sd[pp].x += (double)Sf[pp].x;
                Sd[pp].y += (double)Sf[pp].y;
                Sf[pp] = make_float2(0.f, 0.f);
            }
        }
        if (aborted) break;
        git += cnt;
        mycnt += icnt;
#pragma unroll
        for (int pp = 0; pp < L_PP; ++pp) {
            const int l = 2 * (pp * L_THREADS + tid);
            *reinterpret_cast<float4 *>(part1 + (int64_t)item * PT + l) =
                make_float4(M[pp].x, (float)Sd[pp].x, M[pp].y, (float)Sd[pp].y);
        }
        __syncthreads();
    }
    atomicAdd(&s_pairs, mycnt);
    __syncthreads();
    if (tid == 0) {
        if (s_pairs) atomicAdd(pairs, s_pairs);
        if (aborted) {   // bounded drain of copies that may still be in flight
            for (int s = 0; s < 2; ++s) (void)mbar_wait(&full[s], 0u), (void)mbar_wait(&full[s], 1u);
        }
    }
}


// -------------------------------------------------- tensor-core truncated passes
// The pair exponents come from the mma of rsot_tc.cuh (bitwise the same in
// both passes).  A block pair -- 16 points x 8 targets in pass 1, 16 targets x
// 8 points in pass 2 -- is classified by the bounding balls of its blocks and
// the ranges of the cutoffs of their members:
// "outside" (every pair farther than the radius: skipped), "inside" (every
// pair nearer: no test) or "boundary" (each pair tested, r_qj - b_j > A_q, in
// FP32 on the mma result, as the weight of tp_incl).  The classification margins (1e-4 R) exceed the
// rounding of the pairwise test, so a classified pair gets the decision the
// test would give and both passes sum over the same pairs.

// The per-pair test of a boundary block, on the FMA pipe.  A pair is kept when
// its test value v = r_qj - (b_j - 2k beta_j) exceeds A_q = k|x'_q|^2 - 2k alpha_q;
// y = sat(v 2^64 - A_q 2^64) is one fused multiply-add of v with the exact
// -A_q 2^64 (nAS).  y = 1 for v - A_q >= 2^-64, 0 for v <= A_q, and a fraction
// only for 0 < v - A_q < 2^-64, which needs |v|, |A_q| < 2^-40 (the pair then
// keeps that fraction of its weight).  The weights multiply the exponentials
// (y ex2(e) in one fma), and both passes form v and A_q from the same FP32
// operands, so they weigh every pair alike.
constexpr float TP_S = 18446744073709551616.f;   // 2^64
__device__ __forceinline__ float tp_incl(float v, float nAS) {
    float y;
    asm("fma.rn.sat.f32 %0, %1, %2, %3;" : "=f"(y) : "f"(v), "f"(TP_S), "f"(nAS));
    return y;
}

// exponents and weights of one block pair (pass 1: rows = points with shifts
// ng / ng8 and the scaled tests nAS / nAS8 of rows g / g + 8); y = 1 for the
// pairs of an inside block (bnd false)
__device__ __forceinline__ void tp_lse_pair(const unsigned (&a)[4], uint2 bf, bool bnd, float2 ng,
                                            float2 ng8, float2 nbb, float nAS, float nAS8, float2 &e01,
                                            float2 &e23, float2 &y01, float2 &y23) {
    float d[4];
    mma_tc(d, a, bf);
    e01 = __fadd2_rn(make_float2(d[0], d[1]), ng);
    e23 = __fadd2_rn(make_float2(d[2], d[3]), ng8);
    y01 = y23 = make_float2(1.f, 1.f);
    if (bnd) {
        const float2 v01 = __fadd2_rn(make_float2(d[0], d[1]), nbb);
        const float2 v23 = __fadd2_rn(make_float2(d[2], d[3]), nbb);
        y01 = make_float2(tp_incl(v01.x, nAS), tp_incl(v01.y, nAS));
        y23 = make_float2(tp_incl(v23.x, nAS8), tp_incl(v23.y, nAS8));
    }
}

// the pass-1 epilogue of one block pair on its mma result d: acc (rows g, g + 8)
// += y ex2(d - M); cnt += the weights of a boundary block.  An excluded pair
// whose exponential overflows gives inf * 0 = NaN, which the caller's check
// sends to the exact redo.
__device__ __forceinline__ void tp_lse_epi(const float (&d)[4], bool bnd, float2 ng, float2 ng8,
                                           float2 nbb, float nAS, float nAS8, float2 &acc, float2 &cnt) {
    const float2 e01 = __fadd2_rn(make_float2(d[0], d[1]), ng);
    const float2 e23 = __fadd2_rn(make_float2(d[2], d[3]), ng8);
    const float2 p0 = make_float2(ex2_approx(e01.x), ex2_approx(e23.x));
    const float2 p1 = make_float2(ex2_approx(e01.y), ex2_approx(e23.y));
    if (bnd) {
        const float2 v01 = __fadd2_rn(make_float2(d[0], d[1]), nbb);
        const float2 v23 = __fadd2_rn(make_float2(d[2], d[3]), nbb);
        const float2 y0 = make_float2(tp_incl(v01.x, nAS), tp_incl(v23.x, nAS8));
        const float2 y1 = make_float2(tp_incl(v01.y, nAS), tp_incl(v23.y, nAS8));
        acc = __ffma2_rn(p0, y0, acc);
        acc = __ffma2_rn(p1, y1, acc);
        cnt = __fadd2_rn(cnt, __fadd2_rn(y0, y1));
    } else {
        acc = __fadd2_rn(acc, p0);
        acc = __fadd2_rn(acc, p1);
    }
}

// --------------------------------------------- block-skip tensor-core passes
// The pipeline of the dense tensor-core passes (rsot_dense.cu: 256 threads,
// 4 m-blocks of 16 rows per warp in registers, stages of TC_TS = 1024 records
// in shared memory filled by bulk copies, released per warp on an `empty`
// mbarrier) over the Morton-sorted points and targets, with the truncation:
//   * per CTA, only the stages whose box lies within the largest cutoff
//     radius of the CTA's rows are copied (a box test against the maxima of
//     alpha and beta);
//   * per block pair (16 rows x 8 columns) the class of tp_class: outside
//     pairs skip the mma, boundary pairs test every pair on the mma result.
// Each CTA covers TC_ROWS = 512 rows and one chunk of stages; the partials
// land in the item layout of the queue kernels (items of PT points or TT
// targets, numbered tile * chunks + chunk), so that the same merge kernels
// read them.
constexpr int BS_CHUNK = 8;   // stages per CTA chunk
constexpr size_t BS_SMEM1 =
    (size_t)TC_STAGES * (TC_TS * sizeof(Rec16) + TC_TS * sizeof(float) + TC_NBS * (sizeof(float4) + sizeof(float2)));
constexpr size_t BS_SMEM2 =
    (size_t)TC_STAGES * (TC_TS * sizeof(Rec16) + 2 * TC_TS * sizeof(float) + TC_NBS * (sizeof(float4) + sizeof(float2)));
static_assert(TC_ROWS == 512 && TC_TS == 1024 && PT == 2 * TC_ROWS && TC_ROWS == 2 * TT,
              "block-skip layout: a CTA is half a point tile / two target tiles");

// candidate stages of one CTA: box of its rows (6 floats) and their largest
// alpha / beta against each stage's box and largest beta / alpha
__device__ __forceinline__ int bs_list(const float *__restrict__ rbox, float rmax,
                                       const float *__restrict__ sbox, const float *__restrict__ smax,
                                       int st0, int st1, int *list) {
    float rb[6];
    for (int k = 0; k < 6; ++k) rb[k] = rbox[k];
    int c = 0;
    if (!(rb[0] <= rb[3])) return 0;
    for (int s = st0; s < st1; ++s) {
        float sb[6];
        for (int k = 0; k < 6; ++k) sb[k] = sbox[s * 6 + k];
        if (!(sb[0] <= sb[3])) continue;
        const float rr = sqrtf(fmaxf(0.f, 2.f * (rmax + smax[s]))) * (1.0f + 1e-5f) + 1e-6f;
        if (box_dist2(rb, sb) < rr * rr) list[c++] = s;
    }
    return c;
}

__global__ void __launch_bounds__(TC_THREADS, TC_MINB)
    k_lse_tcb(const Rec16 *__restrict__ prec, const float *__restrict__ Aq,
              const float *__restrict__ M0, const float4 *__restrict__ pball64,
              const float2 *__restrict__ pal64, const float *__restrict__ pbox512,
              const float *__restrict__ pa512, const Rec16 *__restrict__ trec,
              const float *__restrict__ bs, const float4 *__restrict__ tball8,
              const float2 *__restrict__ tbe8, const float *__restrict__ tbox1024,
              const float *__restrict__ tb1024, int nstages, int k1, float2 *__restrict__ part1,
              unsigned long long *__restrict__ pairs, int *__restrict__ flags,
              const int *__restrict__ gate) {
    if (*gate & 1) return;   // operands out of f16 range: the FP32 kernels run
    extern __shared__ __align__(128) unsigned char bs_smem[];
    constexpr size_t oB = TC_STAGES * TC_TS * sizeof(Rec16);
    constexpr size_t oBall = oB + TC_STAGES * TC_TS * sizeof(float);
    constexpr size_t oBe = oBall + TC_STAGES * TC_NBS * sizeof(float4);
    Rec16 (*s_rec)[TC_TS] = reinterpret_cast<Rec16 (*)[TC_TS]>(bs_smem);
    float (*s_b)[TC_TS] = reinterpret_cast<float (*)[TC_TS]>(bs_smem + oB);
    float4 (*s_ball)[TC_NBS] = reinterpret_cast<float4 (*)[TC_NBS]>(bs_smem + oBall);
    float2 (*s_be)[TC_NBS] = reinterpret_cast<float2 (*)[TC_NBS]>(bs_smem + oBe);
    __shared__ __align__(8) uint64_t full[TC_STAGES], empty[TC_STAGES];
    __shared__ int s_list[BS_CHUNK], s_cnt;
    __shared__ unsigned long long s_pairs;
    __shared__ int s_ab;
    constexpr unsigned kStage = TC_TS * (sizeof(Rec16) + sizeof(float)) + TC_NBS * (sizeof(float4) + sizeof(float2));
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, g = lane >> 2, t = lane & 3;
    const int kc = blockIdx.y;
    if (tid == 0) {
        s_cnt = bs_list(pbox512 + (size_t)blockIdx.x * 6, pa512[blockIdx.x], tbox1024, tb1024,
                        kc * BS_CHUNK, min(nstages, (kc + 1) * BS_CHUNK), s_list);
        s_pairs = 0;
        s_ab = 0;
        for (int st = 0; st < TC_STAGES; ++st) {
            mbar_init(&full[st], 1);
            mbar_init(&empty[st], TC_WARPS);
        }
        fence_barrier_init();
    }
    __syncthreads();
    const int cnt = s_cnt;
#define BS_ISSUE1(it_)                                                                               \
    do {                                                                                             \
        const int sl_ = (it_) % TC_STAGES;                                                           \
        const int64_t j_ = (int64_t)s_list[it_] * TC_TS;                                             \
        mbar_expect_tx(&full[sl_], kStage);                                                          \
        bulk_g2s(s_rec[sl_], trec + j_, TC_TS * sizeof(Rec16), &full[sl_]);                          \
        bulk_g2s(s_b[sl_], bs + j_, TC_TS * sizeof(float), &full[sl_]);                              \
        bulk_g2s(s_ball[sl_], tball8 + j_ / 8, TC_NBS * sizeof(float4), &full[sl_]);                 \
        bulk_g2s(s_be[sl_], tbe8 + j_ / 8, TC_NBS * sizeof(float2), &full[sl_]);                     \
    } while (0)
    if (tid == 0)
        for (int it = 0; it < TC_STAGES && it < cnt; ++it) BS_ISSUE1(it);
    int issued = min(TC_STAGES, cnt);
    const int64_t q0 = (int64_t)blockIdx.x * TC_ROWS + warp * (TC_MB * 16);
    const uint2 *pr = reinterpret_cast<const uint2 *>(prec);
    unsigned A[TC_MB][4];
    float nAS[TC_MB], nAS8[TC_MB];   // -A_q 2^64 of rows g, g + 8 (tp_incl)
    float2 M[TC_MB], Sf[TC_MB];
    // FP64 sums of the lane (added once per stage) in shared memory
    __shared__ double2 s_Sd[TC_WARPS][32][TC_MB];
    double2 (&Sd)[TC_MB] = s_Sd[warp][lane];
    unsigned rvs = 0;   // real rows of this lane (rows g, g + 8 of the 4 m-blocks; padding has A = +inf)
#pragma unroll
    for (int m = 0; m < TC_MB; ++m) {
        const int64_t qb = q0 + m * 16;
        tc_load_a(A[m], pr + qb * 4, g, t);
        const float ag = Aq[qb + g], ag8 = Aq[qb + g + 8];
        nAS[m] = ag * -TP_S;
        nAS8[m] = ag8 * -TP_S;
        rvs += (unsigned)(ag < INFINITY) + (unsigned)(ag8 < INFINITY);
        M[m] = make_float2(M0[qb + g], M0[qb + g + 8]);
        Sf[m] = make_float2(0.f, 0.f);
        Sd[m] = make_double2(0.0, 0.0);
    }
    // the warp's 64 rows are classified together against each n-block
    const float4 wball = pball64[q0 / 64];
    const float2 wal = pal64[q0 / 64];
    unsigned icnt = 0;    // pairs of inside blocks
    float2 cntf = make_float2(0.f, 0.f);   // weights of boundary-block pairs (<= 2^14 a lane)
    bool aborted = false;
    for (int it = 0; it < cnt; ++it) {
        const int slot = it % TC_STAGES;
        const unsigned ph = (unsigned)(it / TC_STAGES) & 1u;
        if (!__all_sync(0xffffffffu, mbar_wait(&full[slot], ph))) {
            atomicOr(flags, kErrTimeout);
            aborted = true;
            break;
        }
        {
            const uint2 *rec = reinterpret_cast<const uint2 *>(&s_rec[slot][0]) + lane;
            const float2 *bp = reinterpret_cast<const float2 *>(&s_b[slot][0]) + t;
            // classes of the warp's 64 rows against n-blocks lane + 32 i (2 bits at 2 i)
            unsigned cls = 0;
#pragma unroll
            for (int i = 0; i < 4; ++i)
                cls |= (unsigned)tp_class(wball, s_ball[slot][lane + 32 * i], wal, s_be[slot][lane + 32 * i]) << (2 * i);
#pragma unroll 1
            for (int i = 0; i < 4; ++i) {
                // n-blocks 32 i + l: live (class 1 or 2) and boundary (class 2) bit maps
                const unsigned lvi = __ballot_sync(0xffffffffu, ((cls >> (2 * i)) & 3u) != 0u);
                const unsigned bmi = __ballot_sync(0xffffffffu, ((cls >> (2 * i)) & 3u) == 2u);
#pragma unroll 1
                for (int gq = 0; gq < 32 / TC_GROUP; ++gq) {
                    const int grp = i * (32 / TC_GROUP) + gq;
                    const unsigned gmask = (lvi >> (gq * TC_GROUP)) & 0xffu;
                    if (!gmask) continue;
                    const unsigned bmask = (bmi >> (gq * TC_GROUP)) & 0xffu;
                    float2 acc[TC_MB], ng[TC_MB], ng8[TC_MB];
#pragma unroll
                    for (int m = 0; m < TC_MB; ++m) {
                        acc[m] = make_float2(0.f, 0.f);
                        ng[m] = make_float2(-M[m].x, -M[m].x);
                        ng8[m] = make_float2(-M[m].y, -M[m].y);
                    }
                    for (unsigned gm = gmask; gm;) {
                        const int b0 = __ffs(gm) - 1;
                        gm &= gm - 1;
                        const bool two = gm != 0;
                        const int b1 = two ? __ffs(gm) - 1 : b0;
                        if (two) gm &= gm - 1;
                        const int nb0 = grp * TC_GROUP + b0, nb1 = grp * TC_GROUP + b1;
                        const bool x0 = (bmask >> b0) & 1u, x1 = (bmask >> b1) & 1u;
                        const uint2 bf0 = rec[32 * nb0], bf1 = rec[32 * nb1];
                        float d0[TC_MB][4], d1[TC_MB][4];
#pragma unroll
                        for (int m = 0; m < TC_MB; ++m) {
                            mma_tc(d0[m], A[m], bf0);
                            if (two) mma_tc(d1[m], A[m], bf1);
                        }
#pragma unroll
                        for (int h = 0; h < 2; ++h) {
                            if (h && !two) break;
                            const bool bnd = h ? x1 : x0;
                            const float2 bb = bp[4 * (h ? nb1 : nb0)];
                            const float2 nbb = make_float2(-bb.x, -bb.y);
                            if (!bnd) icnt += rvs * ((unsigned)(bb.x < INFINITY) + (unsigned)(bb.y < INFINITY));
#pragma unroll
                            for (int m = 0; m < TC_MB; ++m)
                                tp_lse_epi(h ? d1[m] : d0[m], bnd, ng[m], ng8[m], nbb, nAS[m], nAS8[m], acc[m], cntf);
                        }
                    }
                    bool bad = false;
#pragma unroll
                    for (int m = 0; m < TC_MB; ++m)
                        bad = bad || !(acc[m].x <= TC_BIG) || !(acc[m].y <= TC_BIG) ||
                              (M[m].x == -INFINITY && acc[m].x != 0.f) || (M[m].y == -INFINITY && acc[m].y != 0.f);
                    if (__any_sync(0xffffffffu, bad)) {
                        // exact redo of the group: maximum over the kept pairs (weight > 0),
                        // shifts raised, sums recomputed (pairs are not counted again)
#pragma unroll
                        for (int m = 0; m < TC_MB; ++m) {
                            float mg = -INFINITY, mg8 = -INFINITY;
                            const float2 z = make_float2(0.f, 0.f);
                            for (unsigned gm = gmask; gm; gm &= gm - 1) {
                                const int b = __ffs(gm) - 1, nb = grp * TC_GROUP + b;
                                const float2 bb = bp[4 * nb];
                                float2 e01, e23, y01, y23;
                                tp_lse_pair(A[m], rec[32 * nb], (bmask >> b) & 1u, z, z, make_float2(-bb.x, -bb.y),
                                            nAS[m], nAS8[m], e01, e23, y01, y23);
                                mg = max3f(mg, y01.x > 0.f ? e01.x : -INFINITY, y01.y > 0.f ? e01.y : -INFINITY);
                                mg8 = max3f(mg8, y23.x > 0.f ? e23.x : -INFINITY, y23.y > 0.f ? e23.y : -INFINITY);
                            }
                            if (mg > -INFINITY) tc_raise(M[m].x, mg, Sf[m].x, Sd[m].x);
                            if (mg8 > -INFINITY) tc_raise(M[m].y, mg8, Sf[m].y, Sd[m].y);
                            const float2 g1 = make_float2(-M[m].x, -M[m].x), g8 = make_float2(-M[m].y, -M[m].y);
                            float2 a2 = make_float2(0.f, 0.f);
                            for (unsigned gm = gmask; gm; gm &= gm - 1) {
                                const int b = __ffs(gm) - 1, nb = grp * TC_GROUP + b;
                                const float2 bb = bp[4 * nb];
                                float2 e01, e23, y01, y23;
                                tp_lse_pair(A[m], rec[32 * nb], (bmask >> b) & 1u, g1, g8, make_float2(-bb.x, -bb.y),
                                            nAS[m], nAS8[m], e01, e23, y01, y23);
                                a2.x += (y01.x > 0.f ? y01.x * ex2_approx(e01.x) : 0.f) +
                                        (y01.y > 0.f ? y01.y * ex2_approx(e01.y) : 0.f);
                                a2.y += (y23.x > 0.f ? y23.x * ex2_approx(e23.x) : 0.f) +
                                        (y23.y > 0.f ? y23.y * ex2_approx(e23.y) : 0.f);
                            }
                            acc[m] = a2;
                        }
                    }
#pragma unroll
                    for (int m = 0; m < TC_MB; ++m) Sf[m] = __fadd2_rn(Sf[m], acc[m]);
                }
            }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[slot]);
        if (warp == 0 && it + TC_STAGES < cnt) {
            bool ok = true;
            if (tid == 0) {
                ok = mbar_wait(&empty[slot], ph);
                if (ok) {
                    BS_ISSUE1(it + TC_STAGES);
                    ++issued;
                }
            }
            if (!__shfl_sync(0xffffffffu, ok, 0)) {
                atomicOr(flags, kErrTimeout);
                aborted = true;
                break;
            }
        }
#pragma unroll
        for (int m = 0; m < TC_MB; ++m) {
            Sd[m].x += (double)Sf[m].x;
            Sd[m].y += (double)Sf[m].y;
            Sf[m] = make_float2(0.f, 0.f);
        }
    }
#undef BS_ISSUE1
    // a warp whose wait expired writes nothing (the error flag is set) but still
    // reaches the closing barrier; thread 0 then drains its copies (bounded)
    if (aborted && lane == 0) s_ab = 1;
    // merge the 4 lanes of each row (common shift = their maximum); item layout
    float2 *o = part1 + ((int64_t)(blockIdx.x >> 1) * k1 + kc) * PT + (blockIdx.x & 1) * TC_ROWS;
#pragma unroll
    for (int m = 0; m < TC_MB && !aborted; ++m) {
        float mx = M[m].x, my = M[m].y;
        mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, 1));
        mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, 2));
        my = fmaxf(my, __shfl_xor_sync(0xffffffffu, my, 1));
        my = fmaxf(my, __shfl_xor_sync(0xffffffffu, my, 2));
        double sx = M[m].x == -INFINITY ? 0.0 : Sd[m].x * pow2_int_d(M[m].x - mx);
        double sy = M[m].y == -INFINITY ? 0.0 : Sd[m].y * pow2_int_d(M[m].y - my);
        sx += __shfl_xor_sync(0xffffffffu, sx, 1);
        sx += __shfl_xor_sync(0xffffffffu, sx, 2);
        sy += __shfl_xor_sync(0xffffffffu, sy, 1);
        sy += __shfl_xor_sync(0xffffffffu, sy, 2);
        if (m == t) {
            const int l = warp * (TC_MB * 16) + m * 16 + g;
            o[l] = mx == -INFINITY ? make_float2(kPadC, 0.f) : make_float2(mx, (float)sx);
            o[l + 8] = my == -INFINITY ? make_float2(kPadC, 0.f) : make_float2(my, (float)sy);
        }
    }
    atomicAdd(&s_pairs, (unsigned long long)icnt + (unsigned long long)__float2uint_rn(cntf.x + cntf.y));
    __syncthreads();
    if (tid == 0) {
        if (s_pairs) atomicAdd(pairs, s_pairs);
        if (s_ab)
            for (int it = 0; it < issued; ++it)
                (void)mbar_wait(&full[it % TC_STAGES], (unsigned)(it / TC_STAGES) & 1u);
    }
}

__global__ void __launch_bounds__(TC_THREADS, TC_MINB)
    k_grad_tcb(const Rec16 *__restrict__ trec, const float *__restrict__ bs,
               const float4 *__restrict__ tball64, const float2 *__restrict__ tbe64,
               const float *__restrict__ tbox512, const float *__restrict__ tb512,
               const Rec16 *__restrict__ prec, const float *__restrict__ us,
               const float *__restrict__ Aq, const float4 *__restrict__ pball8,
               const float2 *__restrict__ pal8, const float *__restrict__ pbox1024,
               const float *__restrict__ pa1024, int nstages, int k2, double *__restrict__ part2,
               int *__restrict__ flags, const int *__restrict__ gate) {
    if (*gate & 1) return;   // operands out of f16 range: the FP32 kernels run
    extern __shared__ __align__(128) unsigned char bs_smem[];
    constexpr size_t oU = TC_STAGES * TC_TS * sizeof(Rec16);
    constexpr size_t oA = oU + TC_STAGES * TC_TS * sizeof(float);
    constexpr size_t oBall = oA + TC_STAGES * TC_TS * sizeof(float);
    constexpr size_t oAl = oBall + TC_STAGES * TC_NBS * sizeof(float4);
    Rec16 (*s_rec)[TC_TS] = reinterpret_cast<Rec16 (*)[TC_TS]>(bs_smem);
    float (*s_u)[TC_TS] = reinterpret_cast<float (*)[TC_TS]>(bs_smem + oU);
    float (*s_A)[TC_TS] = reinterpret_cast<float (*)[TC_TS]>(bs_smem + oA);
    float4 (*s_ball)[TC_NBS] = reinterpret_cast<float4 (*)[TC_NBS]>(bs_smem + oBall);
    float2 (*s_al)[TC_NBS] = reinterpret_cast<float2 (*)[TC_NBS]>(bs_smem + oAl);
    __shared__ __align__(8) uint64_t full[TC_STAGES], empty[TC_STAGES];
    __shared__ int s_list[BS_CHUNK], s_cnt;
    constexpr unsigned kStage = TC_TS * (sizeof(Rec16) + 2 * sizeof(float)) + TC_NBS * (sizeof(float4) + sizeof(float2));
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, g = lane >> 2, t = lane & 3;
    const int kc = blockIdx.y;
    if (tid == 0) {
        s_cnt = bs_list(tbox512 + (size_t)blockIdx.x * 6, tb512[blockIdx.x], pbox1024, pa1024,
                        kc * BS_CHUNK, min(nstages, (kc + 1) * BS_CHUNK), s_list);
        for (int st = 0; st < TC_STAGES; ++st) {
            mbar_init(&full[st], 1);
            mbar_init(&empty[st], TC_WARPS);
        }
        fence_barrier_init();
    }
    __syncthreads();
    const int cnt = s_cnt;
#define BS_ISSUE2(it_)                                                                               \
    do {                                                                                             \
        const int sl_ = (it_) % TC_STAGES;                                                           \
        const int64_t q_ = (int64_t)s_list[it_] * TC_TS;                                             \
        mbar_expect_tx(&full[sl_], kStage);                                                          \
        bulk_g2s(s_rec[sl_], prec + q_, TC_TS * sizeof(Rec16), &full[sl_]);                          \
        bulk_g2s(s_u[sl_], us + q_, TC_TS * sizeof(float), &full[sl_]);                              \
        bulk_g2s(s_A[sl_], Aq + q_, TC_TS * sizeof(float), &full[sl_]);                              \
        bulk_g2s(s_ball[sl_], pball8 + q_ / 8, TC_NBS * sizeof(float4), &full[sl_]);                 \
        bulk_g2s(s_al[sl_], pal8 + q_ / 8, TC_NBS * sizeof(float2), &full[sl_]);                     \
    } while (0)
    if (tid == 0)
        for (int it = 0; it < TC_STAGES && it < cnt; ++it) BS_ISSUE2(it);
    int issued = min(TC_STAGES, cnt);
    const int64_t j0 = (int64_t)blockIdx.x * TC_ROWS + warp * (TC_MB * 16);
    const uint2 *tr = reinterpret_cast<const uint2 *>(trec);
    unsigned A[TC_MB][4];
    float2 bgg[TC_MB], bg8[TC_MB];   // (-b_g, -b_g), (-b_g+8, -b_g+8)
    double2 acc64[TC_MB];
#pragma unroll
    for (int m = 0; m < TC_MB; ++m) {
        const int64_t jb = j0 + m * 16;
        tc_load_a(A[m], tr + jb * 4, g, t);
        const float b0 = bs[jb + g], b8 = bs[jb + g + 8];
        bgg[m] = make_float2(-b0, -b0);
        bg8[m] = make_float2(-b8, -b8);
        acc64[m] = make_double2(0.0, 0.0);
    }
    // the warp's 64 rows are classified together against each n-block
    const float4 wball = tball64[j0 / 64];
    const float2 wbe = tbe64[j0 / 64];
    bool aborted = false;
    for (int it = 0; it < cnt; ++it) {
        const int slot = it % TC_STAGES;
        const unsigned ph = (unsigned)(it / TC_STAGES) & 1u;
        if (!__all_sync(0xffffffffu, mbar_wait(&full[slot], ph))) {
            atomicOr(flags, kErrTimeout);
            aborted = true;
            break;
        }
        {
            const uint2 *rec = reinterpret_cast<const uint2 *>(&s_rec[slot][0]) + lane;
            const float2 *up = reinterpret_cast<const float2 *>(&s_u[slot][0]) + t;
            const float2 *ap = reinterpret_cast<const float2 *>(&s_A[slot][0]) + t;
            float2 acc[TC_MB];
#pragma unroll
            for (int m = 0; m < TC_MB; ++m) acc[m] = make_float2(0.f, 0.f);
            unsigned cls = 0;   // 2 bits at 2 i: n-block lane + 32 i against the warp's 64 rows
#pragma unroll
            for (int i = 0; i < 4; ++i)
                cls |= (unsigned)tp_class(wball, s_ball[slot][lane + 32 * i], wbe, s_al[slot][lane + 32 * i]) << (2 * i);
#pragma unroll 1
            for (int i = 0; i < 4; ++i) {
                const unsigned bmi = __ballot_sync(0xffffffffu, ((cls >> (2 * i)) & 3u) == 2u);
                // two live n-blocks per step (mma of both before either epilogue)
                for (unsigned live = __ballot_sync(0xffffffffu, ((cls >> (2 * i)) & 3u) != 0u); live;) {
                    const int l0 = __ffs(live) - 1;
                    live &= live - 1;
                    const bool two = live != 0;
                    const int l1 = two ? __ffs(live) - 1 : l0;
                    if (two) live &= live - 1;
                    const int nb0 = 32 * i + l0, nb1 = 32 * i + l1;
                    const bool x0 = (bmi >> l0) & 1u, x1 = (bmi >> l1) & 1u;
                    const uint2 bf0 = rec[32 * nb0], bf1 = rec[32 * nb1];
                    float d0[TC_MB][4], d1[TC_MB][4];
#pragma unroll
                    for (int m = 0; m < TC_MB; ++m) {
                        mma_tc(d0[m], A[m], bf0);
                        if (two) mma_tc(d1[m], A[m], bf1);
                    }
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        if (h && !two) break;
                        const int nb = h ? nb1 : nb0;
                        const bool bnd = h ? x1 : x0;
                        const float2 u = up[4 * nb];   // (u_2t, u_2t+1)
                        float2 nAc = make_float2(0.f, 0.f);
                        if (bnd) {
                            const float2 Ac = ap[4 * nb];   // (A_2t, A_2t+1)
                            nAc = make_float2(Ac.x * -TP_S, Ac.y * -TP_S);
                        }
#pragma unroll
                        for (int m = 0; m < TC_MB; ++m) {
                            const float(&d)[4] = h ? d1[m] : d0[m];
                            const float2 e01 = __fadd2_rn(make_float2(d[0], d[1]), u);
                            const float2 e23 = __fadd2_rn(make_float2(d[2], d[3]), u);
                            const float2 p0 = make_float2(ex2_approx(e01.x), ex2_approx(e23.x));
                            const float2 p1 = make_float2(ex2_approx(e01.y), ex2_approx(e23.y));
                            if (bnd) {
                                const float2 v01 = __fadd2_rn(make_float2(d[0], d[1]), bgg[m]);
                                const float2 v23 = __fadd2_rn(make_float2(d[2], d[3]), bg8[m]);
                                acc[m] = __ffma2_rn(p0, make_float2(tp_incl(v01.x, nAc.x), tp_incl(v23.x, nAc.x)), acc[m]);
                                acc[m] = __ffma2_rn(p1, make_float2(tp_incl(v01.y, nAc.y), tp_incl(v23.y, nAc.y)), acc[m]);
                            } else {
                                acc[m] = __fadd2_rn(acc[m], p0);
                                acc[m] = __fadd2_rn(acc[m], p1);
                            }
                        }
                    }
                }
            }
            bool bad = false;
#pragma unroll
            for (int m = 0; m < TC_MB; ++m) bad = bad || !(acc[m].x < INFINITY) || !(acc[m].y < INFINITY);
            if (__any_sync(0xffffffffu, bad)) {
                // an excluded pair whose exponential overflowed (inf * 0): the
                // stage again, with the excluded pairs' exponentials dropped
#pragma unroll
                for (int m = 0; m < TC_MB; ++m) acc[m] = make_float2(0.f, 0.f);
                for (int i = 0; i < 4; ++i) {
                    const unsigned bmi = __ballot_sync(0xffffffffu, ((cls >> (2 * i)) & 3u) == 2u);
                    for (unsigned live = __ballot_sync(0xffffffffu, ((cls >> (2 * i)) & 3u) != 0u); live;
                         live &= live - 1) {
                        const int l = __ffs(live) - 1, nb = 32 * i + l;
                        const bool bnd = (bmi >> l) & 1u;
                        const float2 u = up[4 * nb], Ac = ap[4 * nb];
                        const float2 nAc = make_float2(Ac.x * -TP_S, Ac.y * -TP_S);
#pragma unroll
                        for (int m = 0; m < TC_MB; ++m) {
                            float d[4];
                            mma_tc(d, A[m], rec[32 * nb]);
                            const float e[4] = {d[0] + u.x, d[1] + u.y, d[2] + u.x, d[3] + u.y};
                            const float bg[4] = {bgg[m].x, bgg[m].x, bg8[m].x, bg8[m].x};
                            const float na[4] = {nAc.x, nAc.y, nAc.x, nAc.y};
                            float p[4];
#pragma unroll
                            for (int k = 0; k < 4; ++k) {
                                const float y = bnd ? tp_incl(d[k] + bg[k], na[k]) : 1.f;
                                p[k] = y > 0.f ? y * ex2_approx(e[k]) : 0.f;
                            }
                            acc[m].x += p[0] + p[1];
                            acc[m].y += p[2] + p[3];
                        }
                    }
                }
            }
#pragma unroll
            for (int m = 0; m < TC_MB; ++m) {
                acc64[m].x += (double)acc[m].x;
                acc64[m].y += (double)acc[m].y;
            }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[slot]);
        if (warp == 0 && it + TC_STAGES < cnt) {
            bool ok = true;
            if (tid == 0) {
                ok = mbar_wait(&empty[slot], ph);
                if (ok) {
                    BS_ISSUE2(it + TC_STAGES);
                    ++issued;
                }
            }
            if (!__shfl_sync(0xffffffffu, ok, 0)) {
                atomicOr(flags, kErrTimeout);
                aborted = true;
                break;
            }
        }
    }
#undef BS_ISSUE2
    if (aborted) {
        if (tid == 0)
            for (int it = 0; it < issued; ++it)
                (void)mbar_wait(&full[it % TC_STAGES], (unsigned)(it / TC_STAGES) & 1u);
        return;
    }
#pragma unroll
    for (int m = 0; m < TC_MB; ++m) {
        double x = acc64[m].x, y = acc64[m].y;
        x += __shfl_xor_sync(0xffffffffu, x, 1);
        x += __shfl_xor_sync(0xffffffffu, x, 2);
        y += __shfl_xor_sync(0xffffffffu, y, 1);
        y += __shfl_xor_sync(0xffffffffu, y, 2);
        if (m == t) {
            // target tile of TT: two per CTA; item = tile * k2 + chunk
            const int l = warp * (TC_MB * 16) + m * 16 + g;   // < 512
            const int64_t tile = (int64_t)blockIdx.x * 2 + l / TT;
            double *o = part2 + (tile * k2 + kc) * TT + (l % TT);
            o[0] = x;
            o[8] = y;
        }
    }
}

// ------------------------------------------------- FP32 block-skip passes (FB)
// The block-skip pipeline of the tensor-core truncated passes with the FP32
// exponents of the dense FP32 kernels: r_qj = fma(x0, w0, fma(x1, w1, fma(x2,
// w2, c_j))) in packed FFMA2 over two rows of one lane, bitwise the same in
// both passes (and in the FP32 queue kernels).  A warp owns 128 rows as two
// halves of 64 (lane l: rows 2l, 2l + 1 of each half), each half classified
// by its own ball against every n-block of 8 columns (outside: skipped,
// inside: no test, boundary: the weight tp_incl of every pair), so that both
// halves skip independently.  Per n-block one of three forms: one half live
// (that half's chain alone), both inside (no test), otherwise both halves with
// the weight, each half's class folded into the test's operand.  Stages of
// FB_TS records are bulk-copied into shared memory and released per warp, as
// in the tensor-core passes.
constexpr int FB_THREADS = 256;
constexpr int FB_WARPS = FB_THREADS / 32;
constexpr int FB_ROWS = FB_WARPS * 128;     // rows per CTA
constexpr int FB_TS = TC_TS;                // records per stage (1,024 columns)
constexpr int FB_NBS = FB_TS / 8;           // n-blocks per stage
constexpr int FB_STAGES = 2;
constexpr int FB_GROUP = 8;                 // n-blocks per optimistic group (pass 1)
constexpr size_t FB_SMEM1 = (size_t)FB_STAGES * (FB_TS * sizeof(Rec12) + FB_NBS * (sizeof(float4) + sizeof(float2)));
constexpr size_t FB_SMEM2 =
    (size_t)FB_STAGES * (FB_TS * (sizeof(Rec8) + sizeof(float)) + FB_NBS * (sizeof(float4) + sizeof(float2)));
static_assert(FB_ROWS == PT && FB_TS == 1024 && FB_ROWS % TT == 0, "FB layout: a CTA is a point tile / four target tiles");

// pass-1 exponents of one target for the lane's row pair of half h: returns r
template <int D>
__device__ __forceinline__ float2 fb_r(const float2 (&X)[3], float2 w0, float2 w1, float2 w2, float2 c) {
    float2 r = c;
    if (D == 3) r = __ffma2_rn(X[2], w2, r);
    r = __ffma2_rn(X[1], w1, r);
    r = __ffma2_rn(X[0], w0, r);
    return r;
}

// pass 1, one half of the warp live in an n-block: the eight targets of the
// half's row pair, tested (boundary) or not (inside)
template <int D>
__device__ __forceinline__ void fb1_half(const Rec12 *T, const float2 (&X)[3], float2 ng, float2 a, bool bnd,
                                         float2 &acc, float2 &cntf) {
    if (bnd) {
#pragma unroll
        for (int tt = 0; tt < 8; ++tt) {
            const float4 a4 = T[tt].a, b4 = T[tt].b;
            const float2 r = fb_r<D>(X, make_float2(a4.x, a4.y), make_float2(a4.z, a4.w),
                                     make_float2(b4.x, b4.y), make_float2(b4.z, b4.w));
            const float2 e = __fadd2_rn(r, ng);
            const float2 p = make_float2(ex2_approx(e.x), ex2_approx(e.y));
            const float2 v = __fadd2_rn(r, make_float2(T[tt].c.x, T[tt].c.y));
            const float2 y = make_float2(tp_incl(v.x, a.x), tp_incl(v.y, a.y));
            acc = __ffma2_rn(p, y, acc);
            cntf = __fadd2_rn(cntf, y);
        }
    } else {
#pragma unroll
        for (int tt = 0; tt < 8; ++tt) {
            const float4 a4 = T[tt].a, b4 = T[tt].b;
            const float2 r = fb_r<D>(X, make_float2(a4.x, a4.y), make_float2(a4.z, a4.w),
                                     make_float2(b4.x, b4.y), make_float2(b4.z, b4.w));
            const float2 e = __fadd2_rn(r, ng);
            acc = __fadd2_rn(acc, make_float2(ex2_approx(e.x), ex2_approx(e.y)));
        }
    }
}

template <int D>
__global__ void __launch_bounds__(FB_THREADS, 2)
    k_lse_fb(const float *__restrict__ xs, int64_t nqt, const float *__restrict__ Aq,
             const float *__restrict__ M0, const float4 *__restrict__ pball64,
             const float2 *__restrict__ pal64, const float *__restrict__ pbox1024,
             const float *__restrict__ pa1024, const Rec12 *__restrict__ tdup, int64_t n,
             const float4 *__restrict__ tball8, const float2 *__restrict__ tbe8,
             const float *__restrict__ tbox1024, const float *__restrict__ tb1024, int nstages,
             int k1, float2 *__restrict__ part1, unsigned long long *__restrict__ pairs,
             int *__restrict__ flags) {
    extern __shared__ __align__(128) unsigned char fb_smem[];
    constexpr size_t oBall = (size_t)FB_STAGES * FB_TS * sizeof(Rec12);
    constexpr size_t oBe = oBall + (size_t)FB_STAGES * FB_NBS * sizeof(float4);
    Rec12 (*s_rec)[FB_TS] = reinterpret_cast<Rec12 (*)[FB_TS]>(fb_smem);
    float4 (*s_ball)[FB_NBS] = reinterpret_cast<float4 (*)[FB_NBS]>(fb_smem + oBall);
    float2 (*s_be)[FB_NBS] = reinterpret_cast<float2 (*)[FB_NBS]>(fb_smem + oBe);
    __shared__ __align__(8) uint64_t full[FB_STAGES], empty[FB_STAGES];
    __shared__ int s_list[BS_CHUNK], s_cnt, s_ab;
    __shared__ unsigned long long s_pairs;
    __shared__ double2 s_Sd[FB_WARPS][32][2];
    constexpr unsigned kStage = FB_TS * sizeof(Rec12) + FB_NBS * (sizeof(float4) + sizeof(float2));
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int kc = blockIdx.y;
    if (tid == 0) {
        s_cnt = bs_list(pbox1024 + (size_t)blockIdx.x * 6, pa1024[blockIdx.x], tbox1024, tb1024,
                        kc * BS_CHUNK, min(nstages, (kc + 1) * BS_CHUNK), s_list);
        s_pairs = 0;
        s_ab = 0;
        for (int st = 0; st < FB_STAGES; ++st) {
            mbar_init(&full[st], 1);
            mbar_init(&empty[st], FB_WARPS);
        }
        fence_barrier_init();
    }
    __syncthreads();
    const int cnt = s_cnt;
#define FB_ISSUE1(it_)                                                                               \
    do {                                                                                             \
        const int sl_ = (it_) % FB_STAGES;                                                           \
        const int64_t j_ = (int64_t)s_list[it_] * FB_TS;                                             \
        mbar_expect_tx(&full[sl_], kStage);                                                          \
        bulk_g2s(s_rec[sl_], tdup + j_, FB_TS * sizeof(Rec12), &full[sl_]);                          \
        bulk_g2s(s_ball[sl_], tball8 + j_ / 8, FB_NBS * sizeof(float4), &full[sl_]);                 \
        bulk_g2s(s_be[sl_], tbe8 + j_ / 8, FB_NBS * sizeof(float2), &full[sl_]);                     \
    } while (0)
    if (tid == 0)
        for (int it = 0; it < FB_STAGES && it < cnt; ++it) FB_ISSUE1(it);
    int issued = min(FB_STAGES, cnt);
    const int64_t r0 = (int64_t)blockIdx.x * FB_ROWS + warp * 128;
    float2 X[2][3], M[2], Sf[2], nAS[2];
    unsigned rvs[2];
    float4 wball[2];
    float2 wal[2];
    double2 (&Sd)[2] = s_Sd[warp][lane];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int64_t q = r0 + 64 * h + 2 * lane;
#pragma unroll
        for (int k = 0; k < 3; ++k)
            X[h][k] = k < D ? *reinterpret_cast<const float2 *>(xs + k * nqt + q) : make_float2(0.f, 0.f);
        const float2 A = *reinterpret_cast<const float2 *>(Aq + q);
        nAS[h] = make_float2(A.x * -TP_S, A.y * -TP_S);
        rvs[h] = (unsigned)(A.x < INFINITY) + (unsigned)(A.y < INFINITY);
        M[h] = *reinterpret_cast<const float2 *>(M0 + q);
        Sf[h] = make_float2(0.f, 0.f);
        Sd[h] = make_double2(0.0, 0.0);
        wball[h] = pball64[(r0 + 64 * h) / 64];
        wal[h] = pal64[(r0 + 64 * h) / 64];
    }
    unsigned icnt = 0;                      // pairs of inside blocks (at most 4 rows x 8 stages x FB_TS)
    float2 cntf = make_float2(0.f, 0.f);    // weights of boundary-block pairs
    bool aborted = false;
    for (int it = 0; it < cnt; ++it) {
        const int slot = it % FB_STAGES;
        const unsigned ph = (unsigned)(it / FB_STAGES) & 1u;
        if (!__all_sync(0xffffffffu, mbar_wait(&full[slot], ph))) {
            atomicOr(flags, kErrTimeout);
            aborted = true;
            break;
        }
        // real columns of the stage (FB_TS but in the array's last stage)
        const int sreal = (int)min((int64_t)FB_TS, n - (int64_t)s_list[it] * FB_TS);
        unsigned cls0 = 0, cls1 = 0;   // 2 bits at 2 i: n-block lane + 32 i against half 0 / 1
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const float4 bb = s_ball[slot][lane + 32 * i];
            const float2 be = s_be[slot][lane + 32 * i];
            cls0 |= (unsigned)tp_class(wball[0], bb, wal[0], be) << (2 * i);
            cls1 |= (unsigned)tp_class(wball[1], bb, wal[1], be) << (2 * i);
        }
#pragma unroll 1
        for (int i = 0; i < 4; ++i) {
            const unsigned lv0 = __ballot_sync(0xffffffffu, ((cls0 >> (2 * i)) & 3u) != 0u);
            const unsigned bd0 = __ballot_sync(0xffffffffu, ((cls0 >> (2 * i)) & 3u) == 2u);
            const unsigned lv1 = __ballot_sync(0xffffffffu, ((cls1 >> (2 * i)) & 3u) != 0u);
            const unsigned bd1 = __ballot_sync(0xffffffffu, ((cls1 >> (2 * i)) & 3u) == 2u);
#pragma unroll 1
            for (int gq = 0; gq < 32 / FB_GROUP; ++gq) {
                const int grp = i * (32 / FB_GROUP) + gq;
                const unsigned g0 = (lv0 >> (gq * FB_GROUP)) & 0xffu, g1 = (lv1 >> (gq * FB_GROUP)) & 0xffu;
                if (!(g0 | g1)) continue;
                const unsigned b0 = (bd0 >> (gq * FB_GROUP)) & 0xffu, b1 = (bd1 >> (gq * FB_GROUP)) & 0xffu;
                float2 acc[2], ng[2];
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    acc[h] = make_float2(0.f, 0.f);
                    ng[h] = make_float2(-M[h].x, -M[h].y);
                }
                for (unsigned gm = g0 | g1; gm; gm &= gm - 1) {
                    const int b = __ffs(gm) - 1, nb = grp * FB_GROUP + b;
                    const bool l0 = (g0 >> b) & 1u, l1 = (g1 >> b) & 1u;
                    const bool x0 = (b0 >> b) & 1u, x1 = (b1 >> b) & 1u;
                    const unsigned jreal = (unsigned)max(0, min(8, sreal - 8 * nb));
                    if (l0 && !x0) icnt += rvs[0] * jreal;
                    if (l1 && !x1) icnt += rvs[1] * jreal;
                    const Rec12 *T = &s_rec[slot][8 * nb];
                    if (l0 != l1) {
                        // one half live: its chain alone (eight targets in flight)
                        if (l0) fb1_half<D>(T, X[0], ng[0], nAS[0], x0, acc[0], cntf);
                        else fb1_half<D>(T, X[1], ng[1], nAS[1], x1, acc[1], cntf);
                        continue;
                    }
                    if (l0 && l1 && !x0 && !x1) {
                        // both halves inside: no test, both chains interleaved
#pragma unroll
                        for (int tt = 0; tt < 8; ++tt) {
                            const float4 a4 = T[tt].a, b4 = T[tt].b;
                            const float2 w0 = make_float2(a4.x, a4.y), w1 = make_float2(a4.z, a4.w);
                            const float2 w2 = make_float2(b4.x, b4.y), c = make_float2(b4.z, b4.w);
#pragma unroll
                            for (int h = 0; h < 2; ++h) {
                                const float2 r = fb_r<D>(X[h], w0, w1, w2, c);
                                const float2 e = __fadd2_rn(r, ng[h]);
                                acc[h] = __fadd2_rn(acc[h], make_float2(ex2_approx(e.x), ex2_approx(e.y)));
                            }
                        }
                    } else {
                        // both halves live, at least one on the boundary: per half the weight
                        // tp_incl(v, a) with the half's class folded into a -- its -A 2^64
                        // (boundary: the test), +inf (inside: 1) or -inf (outside: 0) -- so
                        // that every pair takes one form and both chains interleave; the
                        // boundary halves' weights are counted (cb)
                        const float cb0 = x0 ? 1.f : 0.f, cb1 = x1 ? 1.f : 0.f;
                        float2 nAc[2];
#pragma unroll
                        for (int h = 0; h < 2; ++h) {
                            const bool bnd = h ? x1 : x0;
                            const float f = (h ? l1 : l0) ? INFINITY : -INFINITY;
                            nAc[h] = bnd ? nAS[h] : make_float2(f, f);
                        }
#pragma unroll
                        for (int tt = 0; tt < 8; ++tt) {
                            const float4 a4 = T[tt].a, b4 = T[tt].b;
                            const float2 w0 = make_float2(a4.x, a4.y), w1 = make_float2(a4.z, a4.w);
                            const float2 w2 = make_float2(b4.x, b4.y), c = make_float2(b4.z, b4.w);
                            const float2 nbv = make_float2(T[tt].c.x, T[tt].c.y);
#pragma unroll
                            for (int h = 0; h < 2; ++h) {
                                const float2 r = fb_r<D>(X[h], w0, w1, w2, c);
                                const float2 e = __fadd2_rn(r, ng[h]);
                                const float2 p = make_float2(ex2_approx(e.x), ex2_approx(e.y));
                                const float2 v = __fadd2_rn(r, nbv);
                                const float2 y = make_float2(tp_incl(v.x, nAc[h].x), tp_incl(v.y, nAc[h].y));
                                acc[h] = __ffma2_rn(p, y, acc[h]);
                                const float cb = h ? cb1 : cb0;
                                cntf = __ffma2_rn(y, make_float2(cb, cb), cntf);
                            }
                        }
                    }
                }
                bool bad = false;
#pragma unroll
                for (int h = 0; h < 2; ++h)
                    bad = bad || !(acc[h].x <= TC_BIG) || !(acc[h].y <= TC_BIG) ||
                          (M[h].x == -INFINITY && acc[h].x != 0.f) || (M[h].y == -INFINITY && acc[h].y != 0.f);
                if (__any_sync(0xffffffffu, bad)) {
                    // exact redo of the group: maximum over the kept pairs (weight > 0),
                    // shifts raised, sums recomputed (pairs are not counted again)
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const unsigned gh = h ? g1 : g0, bh = h ? b1 : b0;
                        float mx = -INFINITY, my = -INFINITY;
                        for (unsigned gm = gh; gm; gm &= gm - 1) {
                            const int b = __ffs(gm) - 1, nb = grp * FB_GROUP + b;
                            const bool bnd = (bh >> b) & 1u;
                            const Rec12 *T = &s_rec[slot][8 * nb];
                            for (int tt = 0; tt < 8; ++tt) {
                                const float4 a4 = T[tt].a, b4 = T[tt].b;
                                const float2 r = fb_r<D>(X[h], make_float2(a4.x, a4.y), make_float2(a4.z, a4.w),
                                                         make_float2(b4.x, b4.y), make_float2(b4.z, b4.w));
                                float2 y = make_float2(1.f, 1.f);
                                if (bnd) {
                                    const float2 v = __fadd2_rn(r, make_float2(T[tt].c.x, T[tt].c.y));
                                    y = make_float2(tp_incl(v.x, nAS[h].x), tp_incl(v.y, nAS[h].y));
                                }
                                mx = fmaxf(mx, y.x > 0.f ? r.x : -INFINITY);
                                my = fmaxf(my, y.y > 0.f ? r.y : -INFINITY);
                            }
                        }
                        if (mx > -INFINITY) tc_raise(M[h].x, mx, Sf[h].x, Sd[h].x);
                        if (my > -INFINITY) tc_raise(M[h].y, my, Sf[h].y, Sd[h].y);
                        const float2 nm = make_float2(-M[h].x, -M[h].y);
                        float2 a2 = make_float2(0.f, 0.f);
                        for (unsigned gm = gh; gm; gm &= gm - 1) {
                            const int b = __ffs(gm) - 1, nb = grp * FB_GROUP + b;
                            const bool bnd = (bh >> b) & 1u;
                            const Rec12 *T = &s_rec[slot][8 * nb];
                            for (int tt = 0; tt < 8; ++tt) {
                                const float4 a4 = T[tt].a, b4 = T[tt].b;
                                const float2 r = fb_r<D>(X[h], make_float2(a4.x, a4.y), make_float2(a4.z, a4.w),
                                                         make_float2(b4.x, b4.y), make_float2(b4.z, b4.w));
                                float2 y = make_float2(1.f, 1.f);
                                if (bnd) {
                                    const float2 v = __fadd2_rn(r, make_float2(T[tt].c.x, T[tt].c.y));
                                    y = make_float2(tp_incl(v.x, nAS[h].x), tp_incl(v.y, nAS[h].y));
                                }
                                const float2 e = __fadd2_rn(r, nm);
                                a2.x += y.x > 0.f ? y.x * ex2_approx(e.x) : 0.f;
                                a2.y += y.y > 0.f ? y.y * ex2_approx(e.y) : 0.f;
                            }
                        }
                        acc[h] = a2;
                    }
                }
#pragma unroll
                for (int h = 0; h < 2; ++h) Sf[h] = __fadd2_rn(Sf[h], acc[h]);
            }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[slot]);
        if (warp == 0 && it + FB_STAGES < cnt) {
            bool ok = true;
            if (tid == 0) {
                ok = mbar_wait(&empty[slot], ph);
                if (ok) {
                    FB_ISSUE1(it + FB_STAGES);
                    ++issued;
                }
            }
            if (!__shfl_sync(0xffffffffu, ok, 0)) {
                atomicOr(flags, kErrTimeout);
                aborted = true;
                break;
            }
        }
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            Sd[h].x += (double)Sf[h].x;
            Sd[h].y += (double)Sf[h].y;
            Sf[h] = make_float2(0.f, 0.f);
        }
    }
#undef FB_ISSUE1
    if (aborted && lane == 0) s_ab = 1;
    if (!aborted) {
        float2 *o = part1 + ((int64_t)blockIdx.x * k1 + kc) * PT;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int l = warp * 128 + 64 * h + 2 * lane;
            o[l] = M[h].x == -INFINITY ? make_float2(kPadC, 0.f) : make_float2(M[h].x, (float)Sd[h].x);
            o[l + 1] = M[h].y == -INFINITY ? make_float2(kPadC, 0.f) : make_float2(M[h].y, (float)Sd[h].y);
        }
    }
    atomicAdd(&s_pairs, (unsigned long long)icnt + (unsigned long long)__float2uint_rn(cntf.x + cntf.y));
    __syncthreads();
    if (tid == 0) {
        if (s_pairs) atomicAdd(pairs, s_pairs);
        if (s_ab)
            for (int it = 0; it < issued; ++it)
                (void)mbar_wait(&full[it % FB_STAGES], (unsigned)(it / FB_STAGES) & 1u);
    }
}

// sorted point records of the FP32 block-skip pass 2: (x0,x0,x1,x1) (x2,x2,u,u),
// and the points' -A_q 2^64 (the tests' operand, formed once per evaluation)
__global__ void k_pdup_s(const float *__restrict__ xs, const float *__restrict__ u_s,
                         const float *__restrict__ Aq, int64_t nqt, int d, Rec8 *__restrict__ pdup,
                         float *__restrict__ nAq) {
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nqt) return;
    float x[3] = {0.f, 0.f, 0.f};
    for (int t = 0; t < d; ++t) x[t] = xs[t * nqt + q];
    const float u = u_s[q];
    Rec8 r;
    r.a = make_float4(x[0], x[0], x[1], x[1]);
    r.b = make_float4(x[2], x[2], u, u);
    pdup[q] = r;
    nAq[q] = Aq[q] * -TP_S;   // the operand of tp_incl, bitwise as pass 1 forms it
}

// Pass 2: rows are targets (lane l: targets 2l, 2l + 1 of each half of the
// warp's 128), columns the sorted points of the stage; per pair the exponent
// of pass 1 (the same FFMA2 chain on the same operands), shifted by u_q, and
// in boundary blocks weighted by the same tp_incl test.
// pass 2, one half of the warp live in an n-block: the eight points against
// the half's target pair, tested (boundary) or not (inside); Ab holds the
// points' -A_q 2^64
template <int D>
__device__ __forceinline__ void fb2_half(const Rec8 *T, const float *Ab, const float2 (&W)[3], float2 C,
                                         float2 NB, bool bnd, float2 &acc) {
    if (bnd) {
#pragma unroll
        for (int tt = 0; tt < 8; ++tt) {
            const float4 a4 = T[tt].a, b4 = T[tt].b;
            float2 r = C;
            if (D == 3) r = __ffma2_rn(make_float2(b4.x, b4.y), W[2], r);
            r = __ffma2_rn(make_float2(a4.z, a4.w), W[1], r);
            r = __ffma2_rn(make_float2(a4.x, a4.y), W[0], r);
            const float2 e = __fadd2_rn(r, make_float2(b4.z, b4.w));
            const float2 p = make_float2(ex2_approx(e.x), ex2_approx(e.y));
            const float2 v = __fadd2_rn(r, NB);
            const float a = Ab[tt];
            acc = __ffma2_rn(p, make_float2(tp_incl(v.x, a), tp_incl(v.y, a)), acc);
        }
    } else {
#pragma unroll
        for (int tt = 0; tt < 8; ++tt) {
            const float4 a4 = T[tt].a, b4 = T[tt].b;
            float2 r = C;
            if (D == 3) r = __ffma2_rn(make_float2(b4.x, b4.y), W[2], r);
            r = __ffma2_rn(make_float2(a4.z, a4.w), W[1], r);
            r = __ffma2_rn(make_float2(a4.x, a4.y), W[0], r);
            const float2 e = __fadd2_rn(r, make_float2(b4.z, b4.w));
            acc = __fadd2_rn(acc, make_float2(ex2_approx(e.x), ex2_approx(e.y)));
        }
    }
}

template <int D>
__global__ void __launch_bounds__(FB_THREADS, 2)
    k_grad_fb(const Rec12 *__restrict__ tdup, const float4 *__restrict__ tball64,
              const float2 *__restrict__ tbe64, const float *__restrict__ tbox1024,
              const float *__restrict__ tb1024, const Rec8 *__restrict__ pdup,
              const float *__restrict__ nAq, const float4 *__restrict__ pball8,
              const float2 *__restrict__ pal8, const float *__restrict__ pbox1024,
              const float *__restrict__ pa1024, int nstages, int k2, double *__restrict__ part2,
              int *__restrict__ flags) {
    extern __shared__ __align__(128) unsigned char fb_smem[];
    constexpr size_t oA = (size_t)FB_STAGES * FB_TS * sizeof(Rec8);
    constexpr size_t oBall = oA + (size_t)FB_STAGES * FB_TS * sizeof(float);
    constexpr size_t oAl = oBall + (size_t)FB_STAGES * FB_NBS * sizeof(float4);
    Rec8 (*s_rec)[FB_TS] = reinterpret_cast<Rec8 (*)[FB_TS]>(fb_smem);
    float (*s_A)[FB_TS] = reinterpret_cast<float (*)[FB_TS]>(fb_smem + oA);
    float4 (*s_ball)[FB_NBS] = reinterpret_cast<float4 (*)[FB_NBS]>(fb_smem + oBall);
    float2 (*s_al)[FB_NBS] = reinterpret_cast<float2 (*)[FB_NBS]>(fb_smem + oAl);
    __shared__ __align__(8) uint64_t full[FB_STAGES], empty[FB_STAGES];
    __shared__ int s_list[BS_CHUNK], s_cnt;
    constexpr unsigned kStage = FB_TS * (sizeof(Rec8) + sizeof(float)) + FB_NBS * (sizeof(float4) + sizeof(float2));
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int kc = blockIdx.y;
    if (tid == 0) {
        s_cnt = bs_list(tbox1024 + (size_t)blockIdx.x * 6, tb1024[blockIdx.x], pbox1024, pa1024,
                        kc * BS_CHUNK, min(nstages, (kc + 1) * BS_CHUNK), s_list);
        for (int st = 0; st < FB_STAGES; ++st) {
            mbar_init(&full[st], 1);
            mbar_init(&empty[st], FB_WARPS);
        }
        fence_barrier_init();
    }
    __syncthreads();
    const int cnt = s_cnt;
#define FB_ISSUE2(it_)                                                                               \
    do {                                                                                             \
        const int sl_ = (it_) % FB_STAGES;                                                           \
        const int64_t q_ = (int64_t)s_list[it_] * FB_TS;                                             \
        mbar_expect_tx(&full[sl_], kStage);                                                          \
        bulk_g2s(s_rec[sl_], pdup + q_, FB_TS * sizeof(Rec8), &full[sl_]);                           \
        bulk_g2s(s_A[sl_], nAq + q_, FB_TS * sizeof(float), &full[sl_]);                              \
        bulk_g2s(s_ball[sl_], pball8 + q_ / 8, FB_NBS * sizeof(float4), &full[sl_]);                 \
        bulk_g2s(s_al[sl_], pal8 + q_ / 8, FB_NBS * sizeof(float2), &full[sl_]);                     \
    } while (0)
    if (tid == 0)
        for (int it = 0; it < FB_STAGES && it < cnt; ++it) FB_ISSUE2(it);
    int issued = min(FB_STAGES, cnt);
    const int64_t j0 = (int64_t)blockIdx.x * FB_ROWS + warp * 128;
    float2 W[2][3], C[2], NB[2];
    float4 wball[2];
    float2 wbe[2];
    double2 acc64[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int64_t ja = j0 + 64 * h + 2 * lane;
        const Rec12 ra = tdup[ja], rb = tdup[ja + 1];
        W[h][0] = make_float2(ra.a.x, rb.a.x);
        W[h][1] = make_float2(ra.a.z, rb.a.z);
        W[h][2] = make_float2(ra.b.x, rb.b.x);
        C[h] = make_float2(ra.b.z, rb.b.z);
        NB[h] = make_float2(ra.c.x, rb.c.x);
        acc64[h] = make_double2(0.0, 0.0);
        wball[h] = tball64[(j0 + 64 * h) / 64];
        wbe[h] = tbe64[(j0 + 64 * h) / 64];
    }
    bool aborted = false;
    for (int it = 0; it < cnt; ++it) {
        const int slot = it % FB_STAGES;
        const unsigned ph = (unsigned)(it / FB_STAGES) & 1u;
        if (!__all_sync(0xffffffffu, mbar_wait(&full[slot], ph))) {
            atomicOr(flags, kErrTimeout);
            aborted = true;
            break;
        }
        unsigned cls0 = 0, cls1 = 0;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const float4 bb = s_ball[slot][lane + 32 * i];
            const float2 al = s_al[slot][lane + 32 * i];
            cls0 |= (unsigned)tp_class(wball[0], bb, wbe[0], al) << (2 * i);
            cls1 |= (unsigned)tp_class(wball[1], bb, wbe[1], al) << (2 * i);
        }
        float2 acc[2] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
#pragma unroll 1
        for (int i = 0; i < 4; ++i) {
            const unsigned lv0 = __ballot_sync(0xffffffffu, ((cls0 >> (2 * i)) & 3u) != 0u);
            const unsigned bd0 = __ballot_sync(0xffffffffu, ((cls0 >> (2 * i)) & 3u) == 2u);
            const unsigned lv1 = __ballot_sync(0xffffffffu, ((cls1 >> (2 * i)) & 3u) != 0u);
            const unsigned bd1 = __ballot_sync(0xffffffffu, ((cls1 >> (2 * i)) & 3u) == 2u);
            for (unsigned live = lv0 | lv1; live; live &= live - 1) {
                const int b = __ffs(live) - 1, nb = 32 * i + b;
                const bool l0 = (lv0 >> b) & 1u, l1 = (lv1 >> b) & 1u;
                const bool x0 = (bd0 >> b) & 1u, x1 = (bd1 >> b) & 1u;
                const Rec8 *T = &s_rec[slot][8 * nb];
                const float *Ab = &s_A[slot][8 * nb];
                if (l0 != l1) {
                    // one half live: its chain alone (eight points in flight)
                    if (l0) fb2_half<D>(T, Ab, W[0], C[0], NB[0], x0, acc[0]);
                    else fb2_half<D>(T, Ab, W[1], C[1], NB[1], x1, acc[1]);
                    continue;
                }
                if (l0 && l1 && !x0 && !x1) {
                    // both halves inside: no test, both chains interleaved
#pragma unroll
                    for (int tt = 0; tt < 8; ++tt) {
                        const float4 a4 = T[tt].a, b4 = T[tt].b;
                        const float2 x0v = make_float2(a4.x, a4.y), x1v = make_float2(a4.z, a4.w);
                        const float2 x2v = make_float2(b4.x, b4.y), u = make_float2(b4.z, b4.w);
#pragma unroll
                        for (int h = 0; h < 2; ++h) {
                            float2 r = C[h];
                            if (D == 3) r = __ffma2_rn(x2v, W[h][2], r);
                            r = __ffma2_rn(x1v, W[h][1], r);
                            r = __ffma2_rn(x0v, W[h][0], r);
                            const float2 e = __fadd2_rn(r, u);
                            acc[h] = __fadd2_rn(acc[h], make_float2(ex2_approx(e.x), ex2_approx(e.y)));
                        }
                    }
                } else {
                    // both halves live, at least one on the boundary: per half the weight
                    // tp_incl(r + b, -A 2^64) with the half's class folded into b -- its
                    // b'_j (boundary: the test), +inf (inside: 1, or 0 for a padding point,
                    // whose -A 2^64 is -inf) or -inf (outside: 0) -- one form per pair
                    float2 NBc[2];
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const bool bnd = h ? x1 : x0;
                        const float f = (h ? l1 : l0) ? INFINITY : -INFINITY;
                        NBc[h] = bnd ? NB[h] : make_float2(f, f);
                    }
#pragma unroll
                    for (int tt = 0; tt < 8; ++tt) {
                        const float4 a4 = T[tt].a, b4 = T[tt].b;
                        const float2 x0v = make_float2(a4.x, a4.y), x1v = make_float2(a4.z, a4.w);
                        const float2 x2v = make_float2(b4.x, b4.y), u = make_float2(b4.z, b4.w);
                        const float nA = Ab[tt];
#pragma unroll
                        for (int h = 0; h < 2; ++h) {
                            float2 r = C[h];
                            if (D == 3) r = __ffma2_rn(x2v, W[h][2], r);
                            r = __ffma2_rn(x1v, W[h][1], r);
                            r = __ffma2_rn(x0v, W[h][0], r);
                            const float2 e = __fadd2_rn(r, u);
                            const float2 p = make_float2(ex2_approx(e.x), ex2_approx(e.y));
                            const float2 v = __fadd2_rn(r, NBc[h]);
                            const float2 y = make_float2(tp_incl(v.x, nA), tp_incl(v.y, nA));
                            acc[h] = __ffma2_rn(p, y, acc[h]);
                        }
                    }
                }
            }
        }
        bool bad = false;
#pragma unroll
        for (int h = 0; h < 2; ++h) bad = bad || !(acc[h].x < INFINITY) || !(acc[h].y < INFINITY);
        if (__any_sync(0xffffffffu, bad)) {
            // an excluded pair whose exponential overflowed (inf * 0): the stage
            // again, with the excluded pairs' exponentials dropped
#pragma unroll
            for (int h = 0; h < 2; ++h) acc[h] = make_float2(0.f, 0.f);
            for (int i = 0; i < 4; ++i) {
                const unsigned lv0 = __ballot_sync(0xffffffffu, ((cls0 >> (2 * i)) & 3u) != 0u);
                const unsigned bd0 = __ballot_sync(0xffffffffu, ((cls0 >> (2 * i)) & 3u) == 2u);
                const unsigned lv1 = __ballot_sync(0xffffffffu, ((cls1 >> (2 * i)) & 3u) != 0u);
                const unsigned bd1 = __ballot_sync(0xffffffffu, ((cls1 >> (2 * i)) & 3u) == 2u);
                for (unsigned live = lv0 | lv1; live; live &= live - 1) {
                    const int b = __ffs(live) - 1, nb = 32 * i + b;
                    const Rec8 *T = &s_rec[slot][8 * nb];
                    const float *Ab = &s_A[slot][8 * nb];
                    for (int tt = 0; tt < 8; ++tt) {
                        const float4 a4 = T[tt].a, b4 = T[tt].b;
                        const float nA = Ab[tt];
                        for (int h = 0; h < 2; ++h) {
                            if (!(((h ? lv1 : lv0) >> b) & 1u)) continue;
                            const bool bnd = ((h ? bd1 : bd0) >> b) & 1u;
                            float2 r = C[h];
                            if (D == 3) r = __ffma2_rn(make_float2(b4.x, b4.y), W[h][2], r);
                            r = __ffma2_rn(make_float2(a4.z, a4.w), W[h][1], r);
                            r = __ffma2_rn(make_float2(a4.x, a4.y), W[h][0], r);
                            const float2 e = __fadd2_rn(r, make_float2(b4.z, b4.w));
                            float2 y = make_float2(1.f, 1.f);
                            if (bnd) {
                                const float2 v = __fadd2_rn(r, NB[h]);
                                y = make_float2(tp_incl(v.x, nA), tp_incl(v.y, nA));
                            }
                            acc[h].x += y.x > 0.f ? y.x * ex2_approx(e.x) : 0.f;
                            acc[h].y += y.y > 0.f ? y.y * ex2_approx(e.y) : 0.f;
                        }
                    }
                }
            }
        }
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            acc64[h].x += (double)acc[h].x;
            acc64[h].y += (double)acc[h].y;
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[slot]);
        if (warp == 0 && it + FB_STAGES < cnt) {
            bool ok = true;
            if (tid == 0) {
                ok = mbar_wait(&empty[slot], ph);
                if (ok) {
                    FB_ISSUE2(it + FB_STAGES);
                    ++issued;
                }
            }
            if (!__shfl_sync(0xffffffffu, ok, 0)) {
                atomicOr(flags, kErrTimeout);
                aborted = true;
                break;
            }
        }
    }
#undef FB_ISSUE2
    if (aborted) {
        if (tid == 0)
            for (int it = 0; it < issued; ++it)
                (void)mbar_wait(&full[it % FB_STAGES], (unsigned)(it / FB_STAGES) & 1u);
        return;
    }
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int l = warp * 128 + 64 * h + 2 * lane;   // < FB_ROWS; both rows in one target tile
        const int64_t tile = (int64_t)blockIdx.x * (FB_ROWS / TT) + l / TT;
        double *o = part2 + (tile * k2 + kc) * TT + (l % TT);
        o[0] = acc64[h].x;
        o[1] = acc64[h].y;
    }
}

// off[i] = i * k for i <= rows: the item offsets of the block-skip layout
__global__ void k_offsets_uniform(int *__restrict__ off, int rows, int k) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i <= rows) off[i] = i * k;
}

// ------------------------------------------------------------------ combine
// Merge the item partials of each point; write pass-2 point-pair records
// (x0a,x0b,x1a,x1b) (x2a,x2b,ua,ub) (Aa,Ab,0,0); sum m_q eps L_q over the
// points with a non-empty I_q (Algorithm 2 skips the others).
__global__ void k_combine_trunc(const float2 *__restrict__ part1, const int *__restrict__ off1,
                                int64_t nq, int64_t nqt, const float *__restrict__ xs,
                                const double *__restrict__ x64s, const double *__restrict__ mass_s,
                                const double *__restrict__ lm2_s, const float *__restrict__ Aq,
                                const double *__restrict__ psi, double eps, int d,
                                Rec12 *__restrict__ ppair, double *__restrict__ lse_s,
                                double *__restrict__ blockJ, EvalResult *__restrict__ res,
                                float *__restrict__ u_s, const int *__restrict__ gate, int want) {
    // gate: run only when its bit 0 (FP32 fallback) equals `want`
    if (gate && (*gate & 1) != want) return;
    __shared__ double sh[32];
    __shared__ int s_empty;
    if (threadIdx.x == 0) s_empty = 0;
    __syncthreads();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;   // point pair
    double contrib = 0.0;
    int empty = 0;
    if (2 * i < nqt) {
        const double psic = psi[0];
        float x[2][3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}}, u[2] = {kPadC, kPadC}, A[2];
        for (int h = 0; h < 2; ++h) {
            const int64_t q = 2 * i + h;
            A[h] = Aq[q];
            for (int t = 0; t < d; ++t) x[h][t] = xs[t * nqt + q];
            if (q >= nq) continue;
            const int p = (int)(q / PT), l = (int)(q % PT);
            const int a = off1[p], e = off1[p + 1];
            float mx = -INFINITY;
            for (int it = a; it < e; ++it) mx = fmaxf(mx, part1[(int64_t)it * PT + l].x);
            double tot = 0.0;
            for (int it = a; it < e; ++it) {
                const float2 v = part1[(int64_t)it * PT + l];
                if (v.y > 0.f) tot += (double)v.y * pow2_int_d(v.x - mx);
            }
            if (tot > 0.0) {
                const double R = (double)mx + log2(tot);
                lse_s[q] = R;
                if (mass_s[q] > 0.0) {
                    double r2 = 0.0;
                    for (int t = 0; t < d; ++t) r2 += x64s[q * d + t] * x64s[q * d + t];
                    contrib += mass_s[q] * (psic + eps * kLn2 * R - 0.5 * r2);
                    u[h] = (float)fmax(lm2_s[q] - R, -1.0e30);
                }
            } else {
                lse_s[q] = -INFINITY;
                ++empty;
            }
        }
        Rec12 r;
        r.a = make_float4(x[0][0], x[1][0], x[0][1], x[1][1]);
        r.b = make_float4(x[0][2], x[1][2], u[0], u[1]);
        r.c = make_float4(A[0], A[1], 0.f, 0.f);
        ppair[i] = r;
        if (u_s) *reinterpret_cast<float2 *>(u_s + 2 * i) = make_float2(u[0], u[1]);
    }
    if (empty) atomicAdd(&s_empty, empty);
    const double s = block_sum_d(contrib, sh);
    if (threadIdx.x == 0) {
        blockJ[blockIdx.x] = s;
        if (s_empty) atomicAdd(reinterpret_cast<unsigned long long *>(&res->empty), (unsigned long long)s_empty);
    }
}

// ------------------------------------------------------------------- pass 2
template <int D>
__global__ void __launch_bounds__(G_THREADS)
    k_grad_trunc(const Rec12 *__restrict__ ppair, const Rec12 *__restrict__ tdup,
                 const uint32_t *__restrict__ bits_tp, int pw, const int *__restrict__ off2,
                 int ttiles, int ch2, int *__restrict__ counter, double *__restrict__ part2,
                 int *__restrict__ flags, const int *__restrict__ gate = nullptr) {
    if (gate && !(*gate & 1)) return;
    __shared__ __align__(128) Rec12 sm[2][G_STAGE];
    __shared__ __align__(8) uint64_t full[2];
    __shared__ int s_item, s_t, s_cnt, s_abort[2];
    __shared__ int s_list[MAX_CH];
    const int tid = threadIdx.x;
    if (tid == 0) {
        for (int s = 0; s < 2; ++s) mbar_init(&full[s], 1);
        fence_barrier_init();
        s_abort[0] = s_abort[1] = 0;
    }
    __syncthreads();
    const int total = off2[ttiles];
    unsigned git = 0;
    bool aborted = false;
    for (;;) {
        if (tid == 0) {
            const int it = atomicAdd(counter, 1);
            s_item = it;
            if (it < total) {
                const int t = find_row(off2, ttiles, it);
                s_t = t;
                s_cnt = collect_bits(bits_tp + (size_t)t * pw, pw, (it - off2[t]) * ch2, ch2, s_list);
            }
        }
        __syncthreads();
        const int item = s_item;
        if (item >= total) break;
        const int t = s_t;
        const int nst = 2 * s_cnt;   // two stages (512 points each) per point tile
        if (tid == 0) {
            for (int s = 0; s < 2 && s < nst; ++s) {
                const unsigned slot = (git + s) & 1u;
                mbar_expect_tx(&full[slot], G_STAGE * sizeof(Rec12));
                bulk_g2s(sm[slot], ppair + (int64_t)s_list[s >> 1] * (PT / 2) + (s & 1) * G_STAGE,
                         G_STAGE * sizeof(Rec12), &full[slot]);
            }
        }
        float2 W0[G_TPT], W1[G_TPT], W2[G_TPT], C[G_TPT], NB[G_TPT];
        double acc64[G_TPT];
#pragma unroll
        for (int i = 0; i < G_TPT; ++i) {
            const Rec12 r = tdup[(int64_t)t * TT + i * G_THREADS + tid];
            W0[i] = make_float2(r.a.x, r.a.y);
            W1[i] = make_float2(r.a.z, r.a.w);
            W2[i] = make_float2(r.b.x, r.b.y);
            C[i] = make_float2(r.b.z, r.b.w);
            NB[i] = make_float2(r.c.x, r.c.y);
            acc64[i] = 0.0;
        }
        for (int it = 0; it < nst; ++it) {
            const unsigned gs = git + it, slot = gs & 1u, ph = (gs >> 1) & 1u;
            if (!mbar_wait(&full[slot], ph)) {
                s_abort[it & 1] = 1;
                atomicOr(flags, kErrTimeout);
            } else {
                const Rec12 *P = sm[slot];
                float2 acc[G_TPT];
#pragma unroll
                for (int i = 0; i < G_TPT; ++i) acc[i] = make_float2(0.f, 0.f);
#pragma unroll 2
                for (int k = 0; k < G_STAGE; ++k) {
                    const float4 a = P[k].a, b = P[k].b, e = P[k].c;
                    const float2 x0 = make_float2(a.x, a.y), x1 = make_float2(a.z, a.w);
                    const float2 x2 = make_float2(b.x, b.y), u = make_float2(b.z, b.w);
                    const float2 A = make_float2(e.x, e.y);
#pragma unroll
                    for (int i = 0; i < G_TPT; ++i) {
                        float2 r = C[i];
                        if (D == 3) r = __ffma2_rn(x2, W2[i], r);
                        r = __ffma2_rn(x1, W1[i], r);
                        r = __ffma2_rn(x0, W0[i], r);
                        const float2 v = __fadd2_rn(r, NB[i]);
                        const float2 tt = __fadd2_rn(r, u);
                        const float ex = v.x > A.x ? ex2_approx(tt.x) : 0.f;
                        const float ey = v.y > A.y ? ex2_approx(tt.y) : 0.f;
                        acc[i] = __fadd2_rn(acc[i], make_float2(ex, ey));
                    }
                }
#pragma unroll
                for (int i = 0; i < G_TPT; ++i) acc64[i] += (double)acc[i].x + (double)acc[i].y;
            }
            __syncthreads();
            aborted = s_abort[it & 1] != 0;
            if (aborted) break;
            if (tid == 0 && it + 2 < nst) {
                const int s = it + 2;
                mbar_expect_tx(&full[slot], G_STAGE * sizeof(Rec12));
                bulk_g2s(sm[slot], ppair + (int64_t)s_list[s >> 1] * (PT / 2) + (s & 1) * G_STAGE,
                         G_STAGE * sizeof(Rec12), &full[slot]);
            }
        }
        if (aborted) break;
        git += nst;
#pragma unroll
        for (int i = 0; i < G_TPT; ++i) part2[(int64_t)item * TT + i * G_THREADS + tid] = acc64[i];
        __syncthreads();
    }
    if (aborted && tid == 0)
        for (int s = 0; s < 2; ++s) (void)mbar_wait(&full[s], 0u), (void)mbar_wait(&full[s], 1u);
}

__global__ void k_finalize_grad_trunc(const double *__restrict__ part2, const int *__restrict__ off2,
                                      int64_t n, const int *__restrict__ perm_t,
                                      const double *__restrict__ nu_s, double *__restrict__ grad,
                                      const int *__restrict__ gate, int want) {
    if (gate && (*gate & 1) != want) return;
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    const int t = (int)(s / TT), l = (int)(s % TT);
    double g = 0.0;
    for (int it = off2[t]; it < off2[t + 1]; ++it) g += part2[(int64_t)it * TT + l];
    grad[perm_t[s]] = g - nu_s[s];
}

__global__ void k_finalize_J_trunc(const double *__restrict__ blockJ, int nbj,
                                   const double *__restrict__ psinu, int npn,
                                   const double *__restrict__ psi, EvalResult *__restrict__ res) {
    __shared__ double sh[32];
    double a = 0.0, b = 0.0;
    for (int i = threadIdx.x; i < nbj; i += blockDim.x) a += blockJ[i];
    for (int i = threadIdx.x; i < npn; i += blockDim.x) b += psinu[i];
    const double sa = block_sum_d(a, sh);
    const double sb = block_sum_d(b, sh);
    if (threadIdx.x == 0) {
        res->psic = psi[0];
        res->J = sa - sb;
    }
}

// L_q for the caller's point order from the sorted R_q
__global__ void k_point_L_trunc(const double *__restrict__ lse_s, const int *__restrict__ perm_q,
                                const double *__restrict__ x64s, int64_t nq, int d, double eps,
                                const EvalResult *__restrict__ res, double *__restrict__ out) {
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nq) return;
    const double R = lse_s[s];
    double v = -INFINITY;
    if (isfinite(R)) {
        double r2 = 0.0;
        for (int t = 0; t < d; ++t) r2 += x64s[s * d + t] * x64s[s * d + t];
        v = res->psic / eps + kLn2 * R - 0.5 * r2 / eps;
    }
    out[perm_q[s]] = v;
}

int occupancy_of(const void *fn, int threads) {
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, threads, 0) != cudaSuccess || nb < 1)
        nb = 1;
    return nb;
}

cudaError_t sort_keys(unsigned long long *keys, int64_t npow2, cudaStream_t st) {
    const int thr = 256;
    const unsigned blocks = (unsigned)((npow2 + thr - 1) / thr);
    for (int64_t k = 2; k <= npow2; k <<= 1)
        for (int64_t j = k >> 1; j > 0; j >>= 1)
            k_bitonic_step<<<blocks, thr, 0, st>>>(keys, npow2, j, k);
    return cudaGetLastError();
}

int64_t next_pow2(int64_t v) {
    int64_t p = 1;
    while (p < v) p <<= 1;
    return p;
}

}  // namespace

// Build the grid, the sorted copies and the tile boxes (once per problem).
static cudaError_t grid_build(rsot_problem *p) {
    Grid *g = new Grid();
    p->grid = g;
    cudaStream_t st = p->stream;
    cudaError_t e;
    const int d = p->d;
    // common bounding box (translated coordinates), on the host from the FP64 copies
    std::vector<double> hx((size_t)p->nq * d), hy((size_t)p->n * d);
    if ((e = cudaMemcpy(hx.data(), p->x64, hx.size() * 8, cudaMemcpyDeviceToHost))) return e;
    if ((e = cudaMemcpy(hy.data(), p->y64, hy.size() * 8, cudaMemcpyDeviceToHost))) return e;
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (size_t i = 0; i < hx.size(); ++i) {
        lo[i % d] = std::min(lo[i % d], hx[i]);
        hi[i % d] = std::max(hi[i % d], hx[i]);
    }
    for (size_t i = 0; i < hy.size(); ++i) {
        lo[i % d] = std::min(lo[i % d], hy[i]);
        hi[i % d] = std::max(hi[i % d], hy[i]);
    }
    double ext = 0.0;
    for (int k = 0; k < d; ++k) ext = std::max(ext, hi[k] - lo[k]);
    if (!(ext > 0.0)) ext = 1.0;
    const double target_cells = std::max<double>(2.0, (double)std::max(p->nq, p->n) / 2.0);
    int b = (int)ceil(log2(target_cells) / d);
    b = std::max(1, std::min(b, d == 3 ? 10 : 15));
    g->b = b;
    g->G = 1 << b;
    g->h = ext / g->G * (1.0 + 1e-9);
    for (int k = 0; k < 3; ++k) g->lo[k] = k < d ? lo[k] : 0.0;

    g->nqt = round_up(p->nq, PT);
    g->nt = round_up(p->n, TC_TS);   // whole stages of the block-skip passes
    g->ptiles = (int)(g->nqt / PT);
    g->ttiles = (int)(g->nt / TT);
    g->tw = (g->ttiles + 31) / 32;
    g->pw = (g->ptiles + 31) / 32;
    g->ch1 = std::min(MAX_CH, std::max(16, (g->ttiles + 31) / 32));
    g->ch2 = std::min(MAX_CH, std::max(16, (g->ptiles + 31) / 32));
    g->items1_max = (int64_t)g->ptiles * ((g->ttiles + g->ch1 - 1) / g->ch1);
    g->items2_max = (int64_t)g->ttiles * ((g->ptiles + g->ch2 - 1) / g->ch2);
    g->nblk_comb = (int)((g->nqt / 2 + 255) / 256);

    const int64_t npq = next_pow2(p->nq), npt = next_pow2(p->n);
    unsigned long long *kq = nullptr, *kt = nullptr;
    if ((e = cudaMalloc(&kq, npq * 8))) return e;
    if ((e = cudaMalloc(&kt, npt * 8))) return e;
    const double inv_h = 1.0 / g->h;
    k_morton_keys<<<(unsigned)((npq + 255) / 256), 256, 0, st>>>(p->x64, p->nq, npq, d, g->lo[0],
                                                                 g->lo[1], g->lo[2], inv_h, g->G, kq);
    k_morton_keys<<<(unsigned)((npt + 255) / 256), 256, 0, st>>>(p->y64, p->n, npt, d, g->lo[0],
                                                                 g->lo[1], g->lo[2], inv_h, g->G, kt);
    if ((e = sort_keys(kq, npq, st))) return e;
    if ((e = sort_keys(kt, npt, st))) return e;

#define ALLOC(ptr, count) \
    if ((e = cudaMalloc(&(ptr), (size_t)(count) * sizeof(*(ptr))))) return e
    ALLOC(g->perm_q, g->nqt);
    ALLOC(g->perm_t, g->nt);
    ALLOC(g->xs, (int64_t)d * g->nqt);
    ALLOC(g->x64, (int64_t)d * g->nqt);
    ALLOC(g->mass, g->nqt);
    ALLOC(g->lm2, g->nqt);
    ALLOC(g->y64, (int64_t)d * g->nt);
    ALLOC(g->nu, g->nt);
    ALLOC(g->lnu, g->nt);
    ALLOC(g->pbox, (int64_t)g->ptiles * 6);
    ALLOC(g->tbox, (int64_t)g->ttiles * 6);
    ALLOC(g->bits_pt, (int64_t)g->ptiles * g->tw);
    ALLOC(g->bits_tp, (int64_t)g->ttiles * g->pw);
    ALLOC(g->cnt1, g->ptiles);
    ALLOC(g->cnt2, g->ttiles);
    ALLOC(g->off1, g->ptiles + 1);
    ALLOC(g->off2, g->ttiles + 1);
    ALLOC(g->counters, 4);
    ALLOC(g->Aq, g->nqt);
    ALLOC(g->tdup, g->nt);
    ALLOC(g->ppair, g->nqt / 2);
    ALLOC(g->part1, g->items1_max * PT);
    ALLOC(g->part2, g->items2_max * TT);
    ALLOC(g->lse_s, g->nqt);
    ALLOC(g->blockJ, g->nblk_comb);
    ALLOC(g->pball64, g->nqt / 64);
    ALLOC(g->pball8, g->nqt / 8);
    ALLOC(g->tball64, g->nt / 64);
    ALLOC(g->tball8, g->nt / 8);
    ALLOC(g->prec_s, g->nqt);
    ALLOC(g->trec_s, g->nt);
    ALLOC(g->b_s, g->nt);
    ALLOC(g->u_s, g->nqt);
    ALLOC(g->pal8, g->nqt / 8);
    ALLOC(g->pal64, g->nqt / 64);
    ALLOC(g->ptmax, g->ptiles);
    ALLOC(g->tbe8, g->nt / 8);
    ALLOC(g->tbe64, g->nt / 64);
    ALLOC(g->ttmax, g->ttiles);
    ALLOC(g->m0_s, g->nqt);
    g->k1b = (int)((g->nt / TC_TS + BS_CHUNK - 1) / BS_CHUNK);
    g->k2b = (int)((g->nqt / TC_TS + BS_CHUNK - 1) / BS_CHUNK);
    ALLOC(g->pbox512, g->nqt / TC_ROWS * 6);
    ALLOC(g->tbox512, g->nt / TC_ROWS * 6);
    ALLOC(g->tbox1024, g->nt / TC_TS * 6);
    ALLOC(g->pa512, g->nqt / TC_ROWS);
    ALLOC(g->tb512, g->nt / TC_ROWS);
    ALLOC(g->tb1024, g->nt / TC_TS);
    ALLOC(g->part1b, (int64_t)g->ptiles * g->k1b * PT);
    ALLOC(g->part2b, (int64_t)g->ttiles * g->k2b * TT);
    ALLOC(g->off1b, g->ptiles + 1);
    ALLOC(g->off2b, g->ttiles + 1);
    ALLOC(g->pdup_s, g->nqt);
    ALLOC(g->nAq_s, g->nqt);
#undef ALLOC
    k_gather_points<<<(unsigned)((g->nqt + 255) / 256), 256, 0, st>>>(
        kq, p->nq, g->nqt, d, p->x64, p->mass, p->lmass2, g->perm_q, g->xs, g->x64, g->mass, g->lm2);
    k_gather_targets<<<(unsigned)((g->nt + 255) / 256), 256, 0, st>>>(
        kt, p->n, g->nt, d, p->y64, p->nu, p->lnu, g->perm_t, g->y64, g->nu, g->lnu);
    k_tile_boxes<<<(g->ptiles + 127) / 128, 128, 0, st>>>(g->x64, p->nq, d, PT, g->ptiles, g->pbox);
    k_tile_boxes<<<(g->ttiles + 127) / 128, 128, 0, st>>>(g->y64, p->n, d, TT, g->ttiles, g->tbox);
    {
        const int n512p = (int)(g->nqt / TC_ROWS), n512t = (int)(g->nt / TC_ROWS), n1024t = (int)(g->nt / TC_TS);
        k_tile_boxes<<<(n512p + 127) / 128, 128, 0, st>>>(g->x64, p->nq, d, TC_ROWS, n512p, g->pbox512);
        k_tile_boxes<<<(n512t + 127) / 128, 128, 0, st>>>(g->y64, p->n, d, TC_ROWS, n512t, g->tbox512);
        k_tile_boxes<<<(n1024t + 127) / 128, 128, 0, st>>>(g->y64, p->n, d, TC_TS, n1024t, g->tbox1024);
        k_offsets_uniform<<<(g->ptiles + 256) / 256, 256, 0, st>>>(g->off1b, g->ptiles, g->k1b);
        k_offsets_uniform<<<(g->ttiles + 256) / 256, 256, 0, st>>>(g->off2b, g->ttiles, g->k2b);
        if ((e = cudaFuncSetAttribute((const void *)k_lse_tcb, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)BS_SMEM1)))
            return e;
        if ((e = cudaFuncSetAttribute((const void *)k_grad_tcb, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)BS_SMEM2)))
            return e;
        const void *fb1 = d == 3 ? (const void *)k_lse_fb<3> : (const void *)k_lse_fb<2>;
        const void *fb2 = d == 3 ? (const void *)k_grad_fb<3> : (const void *)k_grad_fb<2>;
        if ((e = cudaFuncSetAttribute(fb1, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)FB_SMEM1)))
            return e;
        if ((e = cudaFuncSetAttribute(fb2, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)FB_SMEM2)))
            return e;
    }
    k_block_balls<<<(unsigned)((g->nqt / 64 + 127) / 128), 128, 0, st>>>(g->x64, p->nq, d, 64, g->nqt / 64, g->pball64);
    k_block_balls<<<(unsigned)((g->nqt / 8 + 127) / 128), 128, 0, st>>>(g->x64, p->nq, d, 8, g->nqt / 8, g->pball8);
    k_block_balls<<<(unsigned)((g->nt / 64 + 127) / 128), 128, 0, st>>>(g->y64, p->n, d, 64, g->nt / 64, g->tball64);
    k_block_balls<<<(unsigned)((g->nt / 8 + 127) / 128), 128, 0, st>>>(g->y64, p->n, d, 8, g->nt / 8, g->tball8);
    k_point_recs_s<<<(unsigned)((g->nqt + 255) / 256), 256, 0, st>>>(g->xs, g->nqt, d, p->tc_P, g->prec_s);
    if ((e = cudaGetLastError())) return e;
    if ((e = cudaStreamSynchronize(st))) return e;
    cudaFree(kq);
    cudaFree(kt);
    const void *f1 = d == 3 ? (const void *)k_lse_trunc<3> : (const void *)k_lse_trunc<2>;
    const void *f2 = d == 3 ? (const void *)k_grad_trunc<3> : (const void *)k_grad_trunc<2>;
    g->slots1 = p->num_sms * occupancy_of(f1, L_THREADS);
    g->slots2 = p->num_sms * occupancy_of(f2, G_THREADS);
    return cudaSuccess;
}

template <int D>
static cudaError_t trunc_mixed(rsot_problem *p, const double *psi, double eps, double *grad) {
    Grid *g = p->grid;
    cudaStream_t st = p->stream;
    // c(x,y) = |x-y|^2/2 < alpha_q + beta_j  <=>  k |x'-y'|^2 < 2k (alpha_q + beta_j)
    const double k = kLog2e / (2.0 * eps);
    auto nb_of = [](int64_t m) { return (unsigned)((m + 255) / 256); };
    trace_begin(p, "trunc_setup");
    k_trunc_A<<<nb_of(g->nqt), 256, 0, st>>>(g->xs, p->nq, g->nqt, D, (float)k, p->alpha, g->perm_q,
                                             2.0 * k, psi, p->cut_anchored, g->Aq, g->m0_s);
    // cutoff ranges of blocks and tiles (sorted order)
    k_ranges8<<<nb_of(g->nqt / 8), 256, 0, st>>>(p->alpha, g->perm_q, p->nq, g->nqt / 8, g->pal8);
    k_ranges_merge<<<nb_of(g->nqt / 64), 256, 0, st>>>(g->pal8, g->nqt / 8, 8, g->pal64, nullptr, g->nqt / 64);
    k_ranges_merge<<<nb_of(g->ptiles), 256, 0, st>>>(g->pal64, g->nqt / 64, PT / 64, nullptr, g->ptmax,
                                                    g->ptiles);
    k_ranges8<<<nb_of(g->nt / 8), 256, 0, st>>>(p->beta, g->perm_t, p->n, g->nt / 8, g->tbe8);
    k_ranges_merge<<<nb_of(g->nt / 64), 256, 0, st>>>(g->tbe8, g->nt / 8, 8, g->tbe64, nullptr, g->nt / 64);
    k_ranges_merge<<<nb_of(g->ttiles), 256, 0, st>>>(g->tbe64, g->nt / 64, TT / 64, nullptr, g->ttmax,
                                                    g->ttiles);
    k_ranges_merge<<<nb_of(g->nqt / TC_ROWS), 256, 0, st>>>(g->pal64, g->nqt / 64, TC_ROWS / 64, nullptr,
                                                           g->pa512, g->nqt / TC_ROWS);
    k_ranges_merge<<<nb_of(g->nt / TC_ROWS), 256, 0, st>>>(g->tbe64, g->nt / 64, TC_ROWS / 64, nullptr,
                                                          g->tb512, g->nt / TC_ROWS);
    k_ranges_merge<<<nb_of(g->nt / TC_TS), 256, 0, st>>>(g->tbe64, g->nt / 64, TC_TS / 64, nullptr,
                                                        g->tb1024, g->nt / TC_TS);
    cudaMemsetAsync(g->bits_tp, 0, (size_t)g->ttiles * g->pw * 4, st);
    cudaMemsetAsync(g->cnt2, 0, (size_t)g->ttiles * 4, st);
    k_tile_pairs<<<g->ptiles, 256, 0, st>>>(g->pbox, g->tbox, g->ptiles, g->ttiles, g->tw, g->pw,
                                            g->ptmax, g->ttmax, g->bits_pt, g->bits_tp, g->cnt1, g->cnt2);
    k_item_offsets<<<1, 64, 0, st>>>(g->cnt1, g->ptiles, g->ch1, g->cnt2, g->ttiles, g->ch2, g->off1,
                                     g->off2, g->counters);
    const int nbp = (int)((g->nt + 255) / 256);
    // tensor-core passes (the automatic choice of the dense path), FP32 passes as
    // their fallback when an operand leaves the f16 range (gate)
    const bool tc = use_tensor_pairs(p);
    int *gate = tc ? &p->res_dev->gate : nullptr;
    k_prep_trunc<<<nbp, 256, 0, st>>>(psi, g->perm_t, g->y64, g->lnu, p->n, g->nt, D, eps, g->tdup,
                                      p->psinu, g->nu, p->flags, tc ? g->trec_s : nullptr, g->b_s,
                                      1.0 / (double)p->tc_P, gate, p->beta);
    trace_end(p);
    unsigned long long *pairs = reinterpret_cast<unsigned long long *>(&p->res_dev->pairs);
    // block pairs are classified against their members' cutoff radii widened /
    // narrowed by 1e-4 relative: the pairwise FP32 test's rounding is far below
    if (!tc) {
        // FP32 pair arithmetic on the block-skip pipeline
        trace_begin(p, "lse_trunc_fb");
        k_lse_fb<D><<<dim3((unsigned)(g->nqt / FB_ROWS), (unsigned)g->k1b), FB_THREADS, FB_SMEM1, st>>>(
            g->xs, g->nqt, g->Aq, g->m0_s, g->pball64, g->pal64, g->pbox, g->ptmax, g->tdup, p->n,
            g->tball8, g->tbe8, g->tbox1024, g->tb1024, (int)(g->nt / FB_TS), g->k1b, g->part1b, pairs,
            p->flags);
        trace_end(p);
        trace_begin(p, "combine_trunc_mixed");
        k_combine_trunc<<<g->nblk_comb, 256, 0, st>>>(g->part1b, g->off1b, p->nq, g->nqt, g->xs, g->x64,
                                                      g->mass, g->lm2, g->Aq, psi, eps, D, g->ppair,
                                                      g->lse_s, g->blockJ, p->res_dev, g->u_s, nullptr, 0);
        k_pdup_s<<<nb_of(g->nqt), 256, 0, st>>>(g->xs, g->u_s, g->Aq, g->nqt, D, g->pdup_s, g->nAq_s);
        trace_end(p);
        trace_begin(p, "grad_trunc_fb");
        k_grad_fb<D><<<dim3((unsigned)(g->nt / FB_ROWS), (unsigned)g->k2b), FB_THREADS, FB_SMEM2, st>>>(
            g->tdup, g->tball64, g->tbe64, g->tbox1024, g->tb1024, g->pdup_s, g->nAq_s, g->pball8, g->pal8,
            g->pbox, g->ptmax, (int)(g->nqt / FB_TS), g->k2b, g->part2b, p->flags);
        trace_end(p);
        trace_begin(p, "finalize_trunc");
        k_finalize_grad_trunc<<<(unsigned)((p->n + 255) / 256), 256, 0, st>>>(g->part2b, g->off2b, p->n,
                                                                              g->perm_t, g->nu, grad,
                                                                              nullptr, 0);
        k_finalize_J_trunc<<<1, 256, 0, st>>>(g->blockJ, g->nblk_comb, p->psinu, nbp, psi, p->res_dev);
        trace_end(p);
        return cudaGetLastError();
    }
    if (tc) {
        trace_begin(p, "lse_trunc_tc");
        k_lse_tcb<<<dim3((unsigned)(g->nqt / TC_ROWS), (unsigned)g->k1b), TC_THREADS, BS_SMEM1, st>>>(
            g->prec_s, g->Aq, g->m0_s, g->pball64, g->pal64, g->pbox512, g->pa512, g->trec_s, g->b_s,
            g->tball8, g->tbe8, g->tbox1024, g->tb1024, (int)(g->nt / TC_TS), g->k1b, g->part1b, pairs,
            p->flags, gate);
        trace_end(p);
    }
    trace_begin(p, "lse_trunc_mixed");
    k_lse_trunc<D><<<g->slots1, L_THREADS, 0, st>>>(g->xs, g->nqt, g->Aq, g->tdup, g->bits_pt, g->tw,
                                                    g->off1, g->ptiles, g->ch1, g->counters,
                                                    g->part1, pairs, p->flags, gate);
    trace_end(p);
    trace_begin(p, "combine_trunc_mixed");
    if (tc)
        k_combine_trunc<<<g->nblk_comb, 256, 0, st>>>(g->part1b, g->off1b, p->nq, g->nqt, g->xs, g->x64,
                                                      g->mass, g->lm2, g->Aq, psi, eps, D, g->ppair,
                                                      g->lse_s, g->blockJ, p->res_dev, g->u_s, gate, 0);
    k_combine_trunc<<<g->nblk_comb, 256, 0, st>>>(g->part1, g->off1, p->nq, g->nqt, g->xs, g->x64,
                                                  g->mass, g->lm2, g->Aq, psi, eps, D, g->ppair,
                                                  g->lse_s, g->blockJ, p->res_dev,
                                                  tc ? g->u_s : nullptr, gate, 1);
    trace_end(p);
    if (tc) {
        trace_begin(p, "grad_trunc_tc");
        k_grad_tcb<<<dim3((unsigned)(g->nt / TC_ROWS), (unsigned)g->k2b), TC_THREADS, BS_SMEM2, st>>>(
            g->trec_s, g->b_s, g->tball64, g->tbe64, g->tbox512, g->tb512, g->prec_s, g->u_s, g->Aq,
            g->pball8, g->pal8, g->pbox, g->ptmax, (int)(g->nqt / TC_TS), g->k2b, g->part2b, p->flags, gate);
        trace_end(p);
    }
    trace_begin(p, "grad_trunc_mixed");
    k_grad_trunc<D><<<g->slots2, G_THREADS, 0, st>>>(g->ppair, g->tdup, g->bits_tp, g->pw, g->off2,
                                                     g->ttiles, g->ch2, g->counters + 1, g->part2,
                                                     p->flags, gate);
    trace_end(p);
    trace_begin(p, "finalize_trunc");
    if (tc)
        k_finalize_grad_trunc<<<(unsigned)((p->n + 255) / 256), 256, 0, st>>>(g->part2b, g->off2b, p->n,
                                                                              g->perm_t, g->nu, grad, gate, 0);
    k_finalize_grad_trunc<<<(unsigned)((p->n + 255) / 256), 256, 0, st>>>(g->part2, g->off2, p->n,
                                                                          g->perm_t, g->nu, grad, gate, 1);
    k_finalize_J_trunc<<<1, 256, 0, st>>>(g->blockJ, g->nblk_comb, p->psinu, nbp, psi, p->res_dev);
    trace_end(p);
    return cudaGetLastError();
}

cudaError_t trunc_eval(rsot_problem *p, const double *psi, double eps, int mixed, double *grad) {
    if (!mixed) return launch_trunc_fp64(p, psi, eps, grad);
    if (!p->grid) {
        cudaError_t e = grid_build(p);
        if (e) return e;
    }
    // the target prep writes one psi.nu partial per 256 sorted targets
    if ((int64_t)p->nblk_prep * 256 < p->grid->nt) return cudaErrorInvalidValue;
    return p->d == 3 ? trunc_mixed<3>(p, psi, eps, grad) : trunc_mixed<2>(p, psi, eps, grad);
}

cudaError_t trunc_sorted_targets(rsot_problem *p, SortedTargets *out) {
    if (!p->grid) {
        cudaError_t e = grid_build(p);
        if (e) return e;
    }
    if (p->grid->nt != p->n_pad) return cudaErrorInvalidValue;   // both pad to whole 1,024s
    out->perm = p->grid->perm_t;
    out->y64 = p->grid->y64;
    out->ball8 = p->grid->tball8;
    out->ball64 = p->grid->tball64;
    return cudaSuccess;
}

cudaError_t trunc_point_L(rsot_problem *p, double *L) {
    if (p->last_kind != 3 || !p->grid) return launch_point_L(p, L);
    Grid *g = p->grid;
    k_point_L_trunc<<<(unsigned)((p->nq + 255) / 256), 256, 0, p->stream>>>(
        g->lse_s, g->perm_q, g->x64, p->nq, p->d, p->last_eps, p->res_dev, L);
    return cudaGetLastError();
}

void trunc_free(rsot_problem *p) {
    Grid *g = p->grid;
    if (!g) return;
    void *ptrs[] = {g->perm_q, g->perm_t, g->xs, g->x64, g->mass, g->lm2, g->y64, g->nu, g->lnu,
                    g->pbox, g->tbox, g->bits_pt, g->bits_tp, g->cnt1, g->cnt2, g->off1, g->off2,
                    g->counters, g->Aq, g->tdup, g->ppair, g->part1, g->part2, g->lse_s, g->blockJ,
                    g->pball64, g->pball8, g->tball64, g->tball8, g->prec_s, g->trec_s, g->b_s,
                    g->u_s, g->pal8, g->pal64, g->ptmax, g->tbe8, g->tbe64, g->ttmax, g->m0_s,
                    g->pbox512, g->tbox512, g->tbox1024, g->pa512, g->tb512, g->tb1024, g->part1b,
                    g->part2b, g->off1b, g->off2b, g->pdup_s, g->nAq_s};
    for (void *q : ptrs) cudaFree(q);
    delete g;
    p->grid = nullptr;
}

}  // namespace rsot
