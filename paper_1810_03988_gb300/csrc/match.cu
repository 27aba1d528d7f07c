// Feature matching and homography estimation (Sec. 4.2, Algorithm 3) on the GPU: Multi-Probe LSH
// matching of BRIEF descriptors, then PROSAC over the matches in quality order.  Decisions are
// those of the definition in integer arithmetic (hash keys, Hamming distances, ratio test,
// ordering) and in IEEE double without contractions (every double operation below is an explicit
// round-to-nearest intrinsic, evaluated in the order of the definition), so that the PROSAC
// samples, hypotheses, inlier counts and the refit are bit-identical to a sequential evaluation:
//   M1 L tables hashing a descriptor to k given bit positions; a query probes its own bucket and
//      the k buckets at Hamming distance 1 of every table; the nearest probed descriptor (ties to
//      the lower index) is the match when its distance <= max_dist and den * d1 < num * d2 (d2:
//      nearest other probed index, none passes);
//   M2 quality order: distance ascending, query index ascending;
//   M3 PROSAC (Chum and Matas growth schedule, m = 4, T_N = 200000; the newest of the top n plus 3
//      of the top n - 1, or 4 of the top n once t > T'_n, drawn without replacement from given
//      random words); 4-point homography (h33 = 1) by 8x8 Gaussian elimination with partial
//      pivoting in coordinates normalised per image (bounding box of the matched points);
//      inliers: w > 0 and squared transfer error < (inlier_px scaled)^2; best: most inliers,
//      ties to the earlier iteration; least squares on its inliers; returned in pixels.
#include <climits>

#include "stitch_internal.cuh"

namespace {

constexpr int MT_MAX_POINTS = 2048;
constexpr int MT_MAX_TABLES = 32, MT_MAX_BITS = 20;

struct LshBits {
    int L, k;
    uint8_t b[MT_MAX_TABLES][MT_MAX_BITS];
};

struct Norm {
    double ca0, ca1, cb0, cb1, sa, sb;
};

__device__ __forceinline__ double dA(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double dS(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ double dM(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double dD(double a, double b) { return __ddiv_rn(a, b); }

__device__ __forceinline__ unsigned lsh_key(const unsigned* d, const LshBits& lb, int l) {
    unsigned key = 0;
    for (int j = 0; j < lb.k; ++j) {
        const int bit = lb.b[l][j];
        key |= ((d[bit >> 5] >> (bit & 31)) & 1u) << j;
    }
    return key;
}

__device__ __forceinline__ int hamming(const unsigned* a, const unsigned* b) {
    int d = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) d += __popc(a[k] ^ b[k]);
    return d;
}

// one block per table: keys of image B's descriptors, sorted by (key, index)
__global__ void __launch_bounds__(1024) mt_build(const unsigned* __restrict__ desc_b, const int* __restrict__ count_b,
                                                 const __grid_constant__ LshBits lb, unsigned* __restrict__ keys,
                                                 int* __restrict__ ord, int cap) {
    __shared__ unsigned long long e[MT_MAX_POINTS];
    const int l = blockIdx.x, nb = min(*count_b, cap);
    int m = 1;
    while (m < nb) m <<= 1;
    for (int i = threadIdx.x; i < m; i += blockDim.x)
        e[i] = i < nb ? ((unsigned long long)lsh_key(desc_b + 8 * i, lb, l) << 32) | (unsigned)i : ~0ull;
    __syncthreads();
    for (int k = 2; k <= m; k <<= 1)
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < m; i += blockDim.x) {
                const int o = i ^ j;
                if (o <= i) continue;
                const unsigned long long a = e[i], b = e[o];
                if (((i & k) == 0) == (a > b)) {
                    e[i] = b;
                    e[o] = a;
                }
            }
            __syncthreads();
        }
    for (int i = threadIdx.x; i < nb; i += blockDim.x) {
        keys[(size_t)l * cap + i] = (unsigned)(e[i] >> 32);
        ord[(size_t)l * cap + i] = (int)(unsigned)e[i];
    }
}

struct Top2 {
    int d1, b1, d2, b2;
};

__device__ __forceinline__ void top2_add(Top2& t, int d, int b) {
    if (d < t.d1 || (d == t.d1 && b < t.b1)) {
        if (b != t.b1) {
            t.d2 = t.d1;
            t.b2 = t.b1;
        }
        t.d1 = d;
        t.b1 = b;
    } else if (b != t.b1 && (d < t.d2 || (d == t.d2 && b < t.b2))) {
        t.d2 = d;
        t.b2 = b;
    }
}

// a warp per query: lanes take the (table, probe) pairs; (nearest, second nearest other index)
// merged across lanes
__global__ void __launch_bounds__(256) mt_query(const unsigned* __restrict__ desc_a, const int* __restrict__ count_a,
                                                const unsigned* __restrict__ desc_b, const int* __restrict__ count_b,
                                                const __grid_constant__ LshBits lb, const unsigned* __restrict__ keys,
                                                const int* __restrict__ ord, int cap, int max_dist, int rnum, int rden,
                                                int* __restrict__ best) {
    const int a = blockIdx.x * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    const int na = min(*count_a, cap), nb = min(*count_b, cap);
    if (a >= na) return;
    unsigned da[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) da[k] = desc_a[8 * a + k];
    constexpr int INF = 1 << 30;
    Top2 t{INF, -1, INF, -1};
    const int per = lb.k + 1;
    for (int pp = lane; pp < lb.L * per; pp += 32) {
        const int l = pp / per, p = pp - l * per - 1;
        const unsigned q0 = lsh_key(da, lb, l);
        const unsigned q = p < 0 ? q0 : (q0 ^ (1u << p));
        const unsigned* kl = keys + (size_t)l * cap;
        int lo = 0, hi = nb;
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (kl[mid] < q) lo = mid + 1;
            else hi = mid;
        }
        for (int i = lo; i < nb && kl[i] == q; ++i) {
            const int b = ord[(size_t)l * cap + i];
            top2_add(t, hamming(da, desc_b + 8 * b), b);
        }
    }
    // merge: the union's two nearest distinct indices are among the lanes' two nearest
    for (int off = 16; off > 0; off >>= 1) {
        Top2 o;
        o.d1 = __shfl_down_sync(0xffffffffu, t.d1, off);
        o.b1 = __shfl_down_sync(0xffffffffu, t.b1, off);
        o.d2 = __shfl_down_sync(0xffffffffu, t.d2, off);
        o.b2 = __shfl_down_sync(0xffffffffu, t.b2, off);
        if (o.b1 >= 0) top2_add(t, o.d1, o.b1);
        if (o.b2 >= 0) top2_add(t, o.d2, o.b2);
    }
    if (lane == 0) {
        const bool ok = t.b1 >= 0 && t.d1 <= max_dist &&
                        (t.d2 == INF || (long long)rden * t.d1 < (long long)rnum * t.d2);
        best[2 * a] = ok ? t.b1 : -1;
        best[2 * a + 1] = t.d1;
    }
}

// one block: accepted matches in quality order, and the per-image normalisation
__global__ void __launch_bounds__(1024) mt_order(const int* __restrict__ best, const int* __restrict__ count_a, int cap,
                                                 const int* __restrict__ xy_a, const int* __restrict__ xy_b,
                                                 int* __restrict__ matches, int* __restrict__ n_matches,
                                                 Norm* __restrict__ norm) {
    __shared__ unsigned long long e[MT_MAX_POINTS];
    __shared__ int s_n;
    __shared__ int mn[4], mx[4];
    const int na = min(*count_a, cap), t = threadIdx.x;
    if (t == 0) s_n = 0;
    if (t < 4) {
        mn[t] = INT_MAX;
        mx[t] = INT_MIN;
    }
    __syncthreads();
    for (int a = t; a < na; a += blockDim.x)
        if (best[2 * a] >= 0) {
            const int pos = atomicAdd(&s_n, 1);
            e[pos] = ((unsigned long long)best[2 * a + 1] << 32) | (unsigned)a;
        }
    __syncthreads();
    const int n = s_n;
    int m = 1;
    while (m < n) m <<= 1;
    for (int i = n + t; i < m; i += blockDim.x) e[i] = ~0ull;
    __syncthreads();
    for (int k = 2; k <= m; k <<= 1)
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = t; i < m; i += blockDim.x) {
                const int o = i ^ j;
                if (o <= i) continue;
                const unsigned long long a = e[i], b = e[o];
                if (((i & k) == 0) == (a > b)) {
                    e[i] = b;
                    e[o] = a;
                }
            }
            __syncthreads();
        }
    for (int i = t; i < n; i += blockDim.x) {
        const int a = (int)(unsigned)e[i];
        const int b = best[2 * a];
        matches[3 * i] = a;
        matches[3 * i + 1] = b;
        matches[3 * i + 2] = (int)(e[i] >> 32);
        atomicMin(&mn[0], xy_a[2 * a]);
        atomicMax(&mx[0], xy_a[2 * a]);
        atomicMin(&mn[1], xy_a[2 * a + 1]);
        atomicMax(&mx[1], xy_a[2 * a + 1]);
        atomicMin(&mn[2], xy_b[2 * b]);
        atomicMax(&mx[2], xy_b[2 * b]);
        atomicMin(&mn[3], xy_b[2 * b + 1]);
        atomicMax(&mx[3], xy_b[2 * b + 1]);
    }
    __syncthreads();
    if (t == 0) {
        *n_matches = n;
        Norm z{0.0, 0.0, 0.0, 0.0, 1.0, 1.0};
        if (n > 0) {
            z.ca0 = dM(0.5, dA((double)mn[0], (double)mx[0]));
            z.ca1 = dM(0.5, dA((double)mn[1], (double)mx[1]));
            z.cb0 = dM(0.5, dA((double)mn[2], (double)mx[2]));
            z.cb1 = dM(0.5, dA((double)mn[3], (double)mx[3]));
            const int ra = max(mx[0] - mn[0], mx[1] - mn[1]), rb = max(mx[2] - mn[2], mx[3] - mn[3]);
            z.sa = dD(2.0, (double)(ra > 1 ? ra : 1));
            z.sb = dD(2.0, (double)(rb > 1 ? rb : 1));
        }
        *norm = z;
    }
}

__device__ __forceinline__ void norm_pair(const Norm& z, const int* xy_a, const int* xy_b, const int* mt, int i,
                                          double& x, double& y, double& u, double& v) {
    const int a = mt[3 * i], b = mt[3 * i + 1];
    x = dM(dS((double)xy_a[2 * a], z.ca0), z.sa);
    y = dM(dS((double)xy_a[2 * a + 1], z.ca1), z.sa);
    u = dM(dS((double)xy_b[2 * b], z.cb0), z.sb);
    v = dM(dS((double)xy_b[2 * b + 1], z.cb1), z.sb);
}

__device__ bool solve8(double M[8][8], double r[8], double h[8]) {
    for (int c = 0; c < 8; ++c) {
        int p = c;
        for (int i = c + 1; i < 8; ++i)
            if (fabs(M[i][c]) > fabs(M[p][c])) p = i;
        if (!(fabs(M[p][c]) >= 1e-12)) return false;
        if (p != c) {
            for (int j = 0; j < 8; ++j) {
                const double tt = M[c][j];
                M[c][j] = M[p][j];
                M[p][j] = tt;
            }
            const double tt = r[c];
            r[c] = r[p];
            r[p] = tt;
        }
        for (int i = c + 1; i < 8; ++i) {
            const double f = dD(M[i][c], M[c][c]);
            for (int j = c; j < 8; ++j) M[i][j] = dS(M[i][j], dM(f, M[c][j]));
            r[i] = dS(r[i], dM(f, r[c]));
        }
    }
    for (int c = 7; c >= 0; --c) {
        double s = r[c];
        for (int j = c + 1; j < 8; ++j) s = dS(s, dM(M[c][j], h[j]));
        h[c] = dD(s, M[c][c]);
    }
    return true;
}

__device__ __forceinline__ bool inlier(const double h[8], double x, double y, double u, double v, double t2) {
    const double w = dA(dA(dM(h[6], x), dM(h[7], y)), 1.0);
    if (!(w > 0.0)) return false;
    const double pu = dS(dD(dA(dA(dM(h[0], x), dM(h[1], y)), h[2]), w), u);
    const double pv = dS(dD(dA(dA(dM(h[3], x), dM(h[4], y)), h[5]), w), v);
    return dA(dM(pu, pu), dM(pv, pv)) < t2;
}

// the growth schedule (sequential recurrence, one thread)
__global__ void mt_schedule(const int* __restrict__ n_matches, int iters, int* __restrict__ nt,
                            unsigned char* __restrict__ uni) {
    const int N = *n_matches, m = 4;
    if (N < m) return;
    double Tn = 200000.0;
    for (int i = 0; i < m; ++i) Tn = dD(dM(Tn, (double)(m - i)), (double)(N - i));
    int n = m;
    double Tp = 1.0;
    for (int t = 1; t <= iters; ++t) {
        if ((double)t == Tp && n < N) {
            const double Tn1 = dD(dM(Tn, (double)(n + 1)), (double)(n + 1 - m));
            Tp = dA(Tp, ceil(dS(Tn1, Tn)));
            Tn = Tn1;
            n = n + 1;
        }
        nt[t - 1] = n;
        uni[t - 1] = Tp < (double)t ? 1 : 0;
    }
}

__device__ __forceinline__ int nth_free(int j, const int* chosen, int c) {
    int s[4];
    for (int i = 0; i < c; ++i) s[i] = chosen[i];
    for (int i = 1; i < c; ++i)
        for (int k = i; k > 0 && s[k - 1] > s[k]; --k) {
            const int tmp = s[k];
            s[k] = s[k - 1];
            s[k - 1] = tmp;
        }
    for (int i = 0; i < c; ++i)
        if (s[i] <= j) ++j;
    return j;
}

// one thread per iteration: its sample and 4-point hypothesis (valid flag 0 when singular)
__global__ void __launch_bounds__(128) mt_hypotheses(const int* __restrict__ n_matches, int iters,
                                                     const int* __restrict__ nt, const unsigned char* __restrict__ uni,
                                                     const unsigned* __restrict__ rnd, const int* __restrict__ mt,
                                                     const int* __restrict__ xy_a, const int* __restrict__ xy_b,
                                                     const Norm* __restrict__ norm, double* __restrict__ hyp,
                                                     int* __restrict__ valid) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= iters) return;
    valid[t] = 0;
    if (*n_matches < 4) return;
    const Norm z = *norm;
    const int n = nt[t];
    const unsigned* rw = rnd + 4 * (size_t)t;
    int idx[4];
    if (uni[t]) {
        for (int k = 0; k < 4; ++k) idx[k] = nth_free((int)(rw[k] % (unsigned)(n - k)), idx, k);
    } else {
        idx[0] = n - 1;
        int chosen[3];
        for (int k = 0; k < 3; ++k) {
            chosen[k] = nth_free((int)(rw[k] % (unsigned)(n - 1 - k)), chosen, k);
            idx[k + 1] = chosen[k];
        }
    }
    double M[8][8], r[8], h[8];
    for (int k = 0; k < 4; ++k) {
        double x, y, u, v;
        norm_pair(z, xy_a, xy_b, mt, idx[k], x, y, u, v);
        double* m0 = M[2 * k];
        double* m1 = M[2 * k + 1];
        m0[0] = x; m0[1] = y; m0[2] = 1.0; m0[3] = 0.0; m0[4] = 0.0; m0[5] = 0.0; m0[6] = -dM(u, x); m0[7] = -dM(u, y);
        m1[0] = 0.0; m1[1] = 0.0; m1[2] = 0.0; m1[3] = x; m1[4] = y; m1[5] = 1.0; m1[6] = -dM(v, x); m1[7] = -dM(v, y);
        r[2 * k] = u;
        r[2 * k + 1] = v;
    }
    if (!solve8(M, r, h)) return;
    for (int k = 0; k < 8; ++k) hyp[8 * (size_t)t + k] = h[k];
    valid[t] = 1;
}

// one block per hypothesis: its inlier count (-1 when not valid)
__global__ void __launch_bounds__(256) mt_score(const int* __restrict__ n_matches, const double* __restrict__ hyp,
                                                const int* __restrict__ valid, const int* __restrict__ mt,
                                                const int* __restrict__ xy_a, const int* __restrict__ xy_b,
                                                const Norm* __restrict__ norm, double inlier_px,
                                                int* __restrict__ counts) {
    __shared__ int s_c;
    const int t = blockIdx.x;
    if (!valid[t]) {
        if (threadIdx.x == 0) counts[t] = -1;
        return;
    }
    const Norm z = *norm;
    const int nm = *n_matches;
    double h[8];
    for (int k = 0; k < 8; ++k) h[k] = hyp[8 * (size_t)t + k];
    const double tn = dM(inlier_px, z.sb), t2 = dM(tn, tn);
    if (threadIdx.x == 0) s_c = 0;
    __syncthreads();
    int c = 0;
    for (int i = threadIdx.x; i < nm; i += blockDim.x) {
        double x, y, u, v;
        norm_pair(z, xy_a, xy_b, mt, i, x, y, u, v);
        c += inlier(h, x, y, u, v, t2);
    }
    for (int off = 16; off > 0; off >>= 1) c += __shfl_down_sync(0xffffffffu, c, off);
    if ((threadIdx.x & 31) == 0) atomicAdd(&s_c, c);
    __syncthreads();
    if (threadIdx.x == 0) counts[t] = s_c;
}

// one block: the best hypothesis, the inlier flags, the least-squares refit (each normal-equation
// entry summed by one thread over the inliers in quality order), back to pixels
__global__ void __launch_bounds__(256) mt_refit(const int* __restrict__ n_matches, int iters,
                                                const double* __restrict__ hyp, const int* __restrict__ counts,
                                                const int* __restrict__ mt, const int* __restrict__ xy_a,
                                                const int* __restrict__ xy_b, const Norm* __restrict__ norm,
                                                double inlier_px, double* __restrict__ H, int* __restrict__ n_inliers,
                                                unsigned char* __restrict__ inl) {
    __shared__ int s_best, s_cnt;
    __shared__ double Ms[8][8], rs[8];
    const int nm = *n_matches, t = threadIdx.x;
    const Norm z = *norm;
    // best: most inliers, ties to the earliest iteration (a strided scan per thread, then the block)
    __shared__ long long s_red[8];
    long long key = -1;  // (count + 1) << 32 | (2^32 - 1 - t): larger is better
    if (nm >= 4)
        for (int k = t; k < iters; k += blockDim.x) {
            const long long v = ((long long)(counts[k] + 1) << 32) | (long long)(0xffffffffu - (unsigned)k);
            key = v > key ? v : key;
        }
    for (int off = 16; off > 0; off >>= 1) {
        const long long o = __shfl_down_sync(0xffffffffu, key, off);
        key = o > key ? o : key;
    }
    if ((t & 31) == 0) s_red[t >> 5] = key;
    __syncthreads();
    if (t == 0) {
        long long b = s_red[0];
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) b = s_red[w] > b ? s_red[w] : b;
        // an invalid hypothesis (count -1) never wins: key (0 << 32 | .) counts as no model
        s_best = (b >> 32) > 0 ? (int)(0xffffffffu - (unsigned)(b & 0xffffffffll)) : -1;
        s_cnt = (int)(b >> 32) - 1;
        for (int i = 0; i < 9; ++i) H[i] = i % 4 == 0 ? 1.0 : 0.0;
        *n_inliers = 0;
    }
    __syncthreads();
    const int bt = s_best;
    for (int i = t; i < nm; i += blockDim.x) inl[i] = 0;
    if (bt < 0 || s_cnt < 4) return;
    double hb[8];
    for (int k = 0; k < 8; ++k) hb[k] = hyp[8 * (size_t)bt + k];
    const double tn = dM(inlier_px, z.sb), t2 = dM(tn, tn);
    for (int i = t; i < nm; i += blockDim.x) {
        double x, y, u, v;
        norm_pair(z, xy_a, xy_b, mt, i, x, y, u, v);
        inl[i] = inlier(hb, x, y, u, v, t2) ? 1 : 0;
    }
    __syncthreads();
    // entries: 64 of M (p, q) and 8 of r
    if (t < 72) {
        const int p = t < 64 ? t / 8 : t - 64, q = t < 64 ? t % 8 : 0;
        double acc = 0.0;
        for (int i = 0; i < nm; ++i) {
            if (!inl[i]) continue;
            double x, y, u, v;
            norm_pair(z, xy_a, xy_b, mt, i, x, y, u, v);
            const double row0[8] = {x, y, 1.0, 0.0, 0.0, 0.0, -dM(u, x), -dM(u, y)};
            const double row1[8] = {0.0, 0.0, 0.0, x, y, 1.0, -dM(v, x), -dM(v, y)};
            if (t < 64) acc = dA(dA(acc, dM(row0[p], row0[q])), dM(row1[p], row1[q]));
            else acc = dA(dA(acc, dM(row0[p], u)), dM(row1[p], v));
        }
        if (t < 64) Ms[p][q] = acc;
        else rs[p] = acc;
    }
    __syncthreads();
    if (t != 0) return;
    double M[8][8], r[8], h[8];
    for (int p = 0; p < 8; ++p) {
        for (int q = 0; q < 8; ++q) M[p][q] = Ms[p][q];
        r[p] = rs[p];
    }
    const double* hn = solve8(M, r, h) ? h : hb;
    const double Hn[9] = {hn[0], hn[1], hn[2], hn[3], hn[4], hn[5], hn[6], hn[7], 1.0};
    const double Ta[9] = {z.sa, 0.0, -dM(z.sa, z.ca0), 0.0, z.sa, -dM(z.sa, z.ca1), 0.0, 0.0, 1.0};
    const double Tbi[9] = {dD(1.0, z.sb), 0.0, z.cb0, 0.0, dD(1.0, z.sb), z.cb1, 0.0, 0.0, 1.0};
    double P[9], Q[9];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            P[3 * i + j] = dA(dA(dM(Hn[3 * i], Ta[j]), dM(Hn[3 * i + 1], Ta[3 + j])), dM(Hn[3 * i + 2], Ta[6 + j]));
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            Q[3 * i + j] = dA(dA(dM(Tbi[3 * i], P[j]), dM(Tbi[3 * i + 1], P[3 + j])), dM(Tbi[3 * i + 2], P[6 + j]));
    for (int i = 0; i < 9; ++i) H[i] = dD(Q[i], Q[8]);
    *n_inliers = s_cnt;
}

}  // namespace

struct stitch_matcher {
    int device = 0, max_points = 0, max_iters = 0;
    unsigned* keys = nullptr;
    int* ord = nullptr;
    int* best = nullptr;
    Norm* norm = nullptr;
    int* nt = nullptr;
    unsigned char* uni = nullptr;
    double* hyp = nullptr;
    int* valid = nullptr;
    int* counts = nullptr;
};

static void matcher_free(stitch_matcher* c) {
    if (!c) return;
    cudaFree(c->keys);
    cudaFree(c->ord);
    cudaFree(c->best);
    cudaFree(c->norm);
    cudaFree(c->nt);
    cudaFree(c->uni);
    cudaFree(c->hyp);
    cudaFree(c->valid);
    cudaFree(c->counts);
    delete c;
}

extern "C" stitch_status stitch_matcher_create(int32_t max_points, int32_t max_iters, int32_t device,
                                               stitch_matcher** out) {
    if (!out) return STITCH_EINVAL;
    *out = nullptr;
    if (max_points < 1 || max_points > MT_MAX_POINTS || max_iters < 0 || max_iters > (1 << 16)) return STITCH_EINVAL;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess) {
        cudaGetLastError();
        return STITCH_ECUDA;
    }
    if (device < 0 || device >= ndev) return STITCH_EINVAL;
    int prev = -1;
    cudaGetDevice(&prev);
    if (cudaSetDevice(device) != cudaSuccess) return STITCH_ECUDA;
    stitch_matcher* c = new (std::nothrow) stitch_matcher();
    if (!c) return STITCH_ENOMEM;
    c->device = device;
    c->max_points = max_points;
    c->max_iters = max_iters;
    const size_t it = (size_t)std::max(max_iters, 1);
    bool okm = cudaMalloc(&c->keys, sizeof(unsigned) * MT_MAX_TABLES * max_points) == cudaSuccess &&
               cudaMalloc(&c->ord, sizeof(int) * MT_MAX_TABLES * max_points) == cudaSuccess &&
               cudaMalloc(&c->best, sizeof(int) * 2 * max_points) == cudaSuccess &&
               cudaMalloc(&c->norm, sizeof(Norm)) == cudaSuccess && cudaMalloc(&c->nt, sizeof(int) * it) == cudaSuccess &&
               cudaMalloc(&c->uni, it) == cudaSuccess && cudaMalloc(&c->hyp, sizeof(double) * 8 * it) == cudaSuccess &&
               cudaMalloc(&c->valid, sizeof(int) * it) == cudaSuccess &&
               cudaMalloc(&c->counts, sizeof(int) * it) == cudaSuccess;
    if (prev >= 0) cudaSetDevice(prev);
    if (!okm) {
        cudaGetLastError();
        matcher_free(c);
        return STITCH_ENOMEM;
    }
    *out = c;
    return STITCH_OK;
}

extern "C" void stitch_matcher_destroy(stitch_matcher* c) {
    if (!c) return;
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(c->device);
    cudaDeviceSynchronize();
    matcher_free(c);
    if (prev >= 0) cudaSetDevice(prev);
}

extern "C" stitch_status stitch_match_homography(stitch_matcher* c, const int32_t* xy_a, const uint8_t* desc_a,
                                                 const int32_t* count_a, const int32_t* xy_b, const uint8_t* desc_b,
                                                 const int32_t* count_b, const stitch_match_params* prm,
                                                 const uint8_t* bits, const uint32_t* rnd, int32_t* matches,
                                                 int32_t* n_matches, double* H, int32_t* n_inliers, uint8_t* inlier,
                                                 void* stream) {
    if (!c || !xy_a || !desc_a || !count_a || !xy_b || !desc_b || !count_b || !prm || !bits || !matches ||
        !n_matches || !H || !n_inliers || !inlier)
        return STITCH_EINVAL;
    if (prm->tables < 1 || prm->tables > MT_MAX_TABLES || prm->bits < 1 || prm->bits > MT_MAX_BITS ||
        prm->ratio_num < 1 || prm->ratio_den < 1 || prm->iters < 0 || prm->iters > c->max_iters ||
        (prm->iters > 0 && !rnd) || !(prm->inlier_px > 0.0) ||
        ((reinterpret_cast<uintptr_t>(desc_a) | reinterpret_cast<uintptr_t>(desc_b)) & 3) != 0)
        return STITCH_EINVAL;
    LshBits lb{};
    lb.L = prm->tables;
    lb.k = prm->bits;
    for (int l = 0; l < lb.L; ++l)
        for (int j = 0; j < lb.k; ++j) lb.b[l][j] = bits[l * lb.k + j];
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != c->device && cudaSetDevice(c->device) != cudaSuccess) return STITCH_ECUDA;
    cudaStream_t s = (cudaStream_t)stream;
    const int cap = c->max_points;
    const unsigned* da = reinterpret_cast<const unsigned*>(desc_a);
    const unsigned* db = reinterpret_cast<const unsigned*>(desc_b);
    mt_build<<<lb.L, 1024, 0, s>>>(db, count_b, lb, c->keys, c->ord, cap);
    mt_query<<<(cap + 7) / 8, 256, 0, s>>>(da, count_a, db, count_b, lb, c->keys, c->ord, cap, prm->max_dist,
                                           prm->ratio_num, prm->ratio_den, c->best);
    mt_order<<<1, 1024, 0, s>>>(c->best, count_a, cap, xy_a, xy_b, matches, n_matches, c->norm);
    const int iters = prm->iters;
    if (iters > 0) {
        mt_schedule<<<1, 1, 0, s>>>(n_matches, iters, c->nt, c->uni);
        mt_hypotheses<<<(iters + 127) / 128, 128, 0, s>>>(n_matches, iters, c->nt, c->uni, rnd, matches, xy_a, xy_b,
                                                          c->norm, c->hyp, c->valid);
        mt_score<<<iters, 256, 0, s>>>(n_matches, c->hyp, c->valid, matches, xy_a, xy_b, c->norm, prm->inlier_px,
                                       c->counts);
    }
    mt_refit<<<1, 256, 0, s>>>(n_matches, iters, c->hyp, c->counts, matches, xy_a, xy_b, c->norm, prm->inlier_px, H,
                               n_inliers, inlier);
    stitch_status st = cudaGetLastError() == cudaSuccess ? STITCH_OK : STITCH_ECUDA;
    if (prev >= 0 && prev != c->device) cudaSetDevice(prev);
    return st;
}
