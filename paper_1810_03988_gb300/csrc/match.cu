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
//   M3 PROSAC (Chum and Matas growth schedule, m = 4, T_N = 200000, its increments
//      T_{n+1} - T_n evaluated exactly as integer ceilings; the newest of the top n plus 3
//      of the top n - 1, or 4 of the top n once t > T'_n, drawn without replacement from given
//      random words); 4-point homography (h33 = 1) by 8x8 Gaussian elimination with partial
//      pivoting in coordinates normalised per image (bounding box of the matched points);
//      inliers: w > 0 and squared transfer error < (inlier_px scaled)^2; best: most inliers,
//      ties to the earlier iteration; least squares on its inliers; returned in pixels.
//
// Kernels, in launch order: mt_build (a block per table: sorted keys and a radix directory),
// mt_query (a warp per query), mt_order (quality order, bounding boxes), mt_prep (normalised
// coordinates, growth schedule by a block scan), mt_hypotheses_b (a block per iteration: sample and
// 8x8 solve with a thread per matrix entry), mt_score (a block per hypothesis), mt_best (arg-max,
// inlier flags), mt_sums (a warp per normal-equation entry, ordered sums), mt_solve (refit and
// back to pixels).
#include <climits>

#include "stitch_internal.cuh"

namespace {

constexpr int MT_MAX_POINTS = 2048;
constexpr int MT_MAX_TABLES = 32, MT_MAX_BITS = 20;
constexpr int MT_DIR_BITS = 11;                        // radix directory of each sorted table
constexpr int MT_DIR = (1 << MT_DIR_BITS) + 1;

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
                                                 int* __restrict__ ord, int* __restrict__ dir, int cap) {
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
    // directory: dir[v] = first sorted position whose key's top bits are >= v (v = 0..2^D)
    const int D = lb.k < MT_DIR_BITS ? lb.k : MT_DIR_BITS, shift = lb.k - D;
    for (int v = threadIdx.x; v <= (1 << D); v += blockDim.x) {
        const unsigned long long bound = (unsigned long long)v << shift;
        int lo = 0, hi = nb;
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if ((e[mid] >> 32) < bound) lo = mid + 1;
            else hi = mid;
        }
        dir[(size_t)l * MT_DIR + v] = lo;
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
// merged across lanes.  A bucket is located through the table's directory (the range of sorted
// positions whose key has given top bits), then by binary search inside that range.
__global__ void __launch_bounds__(256) mt_query(const unsigned* __restrict__ desc_a, const int* __restrict__ count_a,
                                                const unsigned* __restrict__ desc_b, const int* __restrict__ count_b,
                                                const __grid_constant__ LshBits lb, const unsigned* __restrict__ keys,
                                                const int* __restrict__ ord, const int* __restrict__ dir, int cap,
                                                int max_dist, int rnum, int rden, int* __restrict__ best) {
    const int a = blockIdx.x * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    const int na = min(*count_a, cap), nb = min(*count_b, cap);
    const int shift = lb.k > MT_DIR_BITS ? lb.k - MT_DIR_BITS : 0;
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
        const int* dl = dir + (size_t)l * MT_DIR;
        int lo = dl[q >> shift], hi = dl[(q >> shift) + 1];
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

// |x| of a finite or infinite double orders like its bit pattern read as an integer.
__device__ __forceinline__ long long abs_bits(double x) { return __double_as_longlong(x) & 0x7fffffffffffffffll; }

__device__ __forceinline__ bool inlier(const double h[8], double x, double y, double u, double v, double t2) {
    const double w = dA(dA(dM(h[6], x), dM(h[7], y)), 1.0);
    if (!(w > 0.0)) return false;
    const double pu = dS(dD(dA(dA(dM(h[0], x), dM(h[1], y)), h[2]), w), u);
    const double pv = dS(dD(dA(dA(dM(h[3], x), dM(h[4], y)), h[5]), w), v);
    return dA(dM(pu, pu), dM(pv, pv)) < t2;
}

// one block: the normalised coordinates (x, y, u, v) of every match, and the PROSAC growth
// schedule.  The top n grows to n + 1 at iteration E_j (j = n - 4), E_0 = 1 and E_{j+1} = E_j +
// ceil(T_N m n (n-1) (n-2) / (N (N-1) (N-2) (N-3))) (m = 4, T_N = 200000: the exact increment
// T_{n+1} - T_n of T_n = T_N C(n, m) / C(N, m)), up to n = N; E by a block scan.  For iteration t:
// c = #{j < N - 4 : E_j <= t}, n(t) = 4 + c, uniform sampling when E_c < t.
__global__ void __launch_bounds__(1024) mt_prep(const int* __restrict__ n_matches, const int* __restrict__ mt,
                                                const int* __restrict__ xy_a, const int* __restrict__ xy_b,
                                                const Norm* __restrict__ norm, int iters, double* __restrict__ xyuv,
                                                int* __restrict__ nt, unsigned char* __restrict__ uni) {
    __shared__ long long E[MT_MAX_POINTS];
    __shared__ long long wsum[32];
    const int N = *n_matches, tid = threadIdx.x;
    const Norm z = *norm;
    for (int i = tid; i < N; i += blockDim.x) {
        const int a = mt[3 * i], b = mt[3 * i + 1];
        xyuv[4 * i] = dM(dS((double)xy_a[2 * a], z.ca0), z.sa);
        xyuv[4 * i + 1] = dM(dS((double)xy_a[2 * a + 1], z.ca1), z.sa);
        xyuv[4 * i + 2] = dM(dS((double)xy_b[2 * b], z.cb0), z.sb);
        xyuv[4 * i + 3] = dM(dS((double)xy_b[2 * b + 1], z.cb1), z.sb);
    }
    if (N < 4 || iters == 0) return;
    const int K = N - 4;  // growth events j = 0..K-1 (n = 4 + j)
    const long long Q = (long long)N * (N - 1) * (N - 2) * (N - 3);
    long long d[2] = {0, 0};
    for (int e = 0; e < 2; ++e) {
        const int j = 2 * tid + e;
        if (j < K) {
            const long long n = 4 + j;
            d[e] = (800000LL * n * (n - 1) * (n - 2) + Q - 1) / Q;
        }
    }
    // inclusive scan of the pair sums over the block
    long long v = d[0] + d[1];
    const int lane = tid & 31, w = tid >> 5;
    for (int off = 1; off < 32; off <<= 1) {
        const long long o = __shfl_up_sync(0xffffffffu, v, off);
        if (lane >= off) v += o;
    }
    if (lane == 31) wsum[w] = v;
    __syncthreads();
    if (w == 0) {
        long long x = lane < (int)(blockDim.x >> 5) ? wsum[lane] : 0;
        for (int off = 1; off < 32; off <<= 1) {
            const long long o = __shfl_up_sync(0xffffffffu, x, off);
            if (lane >= off) x += o;
        }
        wsum[lane] = x;
    }
    __syncthreads();
    const long long excl = v - (d[0] + d[1]) + (w > 0 ? wsum[w - 1] : 0);
    // E_j = 1 + sum_{i<j} d_i for j = 0..K
    if (2 * tid <= K) E[2 * tid] = 1 + excl;
    if (2 * tid + 1 <= K) E[2 * tid + 1] = 1 + excl + d[0];
    __syncthreads();
    for (int t = tid + 1; t <= iters; t += blockDim.x) {
        int lo = 0, hi = K;  // c = first j in [0, K) with E_j > t, else K
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (E[mid] <= t) lo = mid + 1;
            else hi = mid;
        }
        nt[t - 1] = 4 + lo;
        uni[t - 1] = E[lo] < t ? 1 : 0;
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

// M h = r on one block (at least 72 threads; every thread calls it): thread (i, j) of the first 72
// holds entry j of row i of A = [M | r] in shared memory and receives the operations of the
// sequential elimination (solve8) in the same order, so h is bit-identical; the pivot search and
// the ordered subtractions of the back substitution run on one thread.  Returns false (on every
// thread) when a pivot is below 1e-12 in magnitude or NaN; h in hs.
struct BlockSolve {
    double A[8][9];
    double hs[8], fv[8], prod[8];
    int piv, sing;
};

__device__ bool solve8_block(BlockSolve& b) {
    const int t = threadIdx.x, i = t / 9, j = t - 9 * (t / 9);
    const bool own = t < 72;
    if (t == 0) b.sing = 0;
    __syncthreads();
    for (int c = 0; c < 8; ++c) {
        if (t == 0) {
            long long bst = abs_bits(b.A[c][c]);
            int p = c;
            for (int k = c + 1; k < 8; ++k) {
                const long long v = abs_bits(b.A[k][c]);
                if (v > bst) {
                    bst = v;
                    p = k;
                }
            }
            b.piv = p;
            if (bst < __double_as_longlong(1e-12) || bst > 0x7ff0000000000000ll) b.sing = 1;
        }
        __syncthreads();
        if (b.sing) return false;
        const int p = b.piv;
        if (p != c && own && i == c && j >= c) {  // columns left of c are never read again
            const double x = b.A[c][j];
            b.A[c][j] = b.A[p][j];
            b.A[p][j] = x;
        }
        __syncthreads();
        if (own && i > c && j == c) b.fv[i] = dD(b.A[i][c], b.A[c][c]);
        __syncthreads();
        if (own && i > c && j >= c) b.A[i][j] = dS(b.A[i][j], dM(b.fv[i], b.A[c][j]));
        __syncthreads();
    }
    for (int c = 7; c >= 0; --c) {
        if (t > c && t < 8) b.prod[t] = dM(b.A[c][t], b.hs[t]);
        __syncthreads();
        if (t == 0) {
            double sacc = b.A[c][8];
            for (int k = c + 1; k < 8; ++k) sacc = dS(sacc, b.prod[k]);
            b.hs[c] = dD(sacc, b.A[c][c]);
        }
        __syncthreads();
    }
    return true;
}

// one block of 96 threads per iteration: its sample and 4-point hypothesis (valid flag 0 when
// singular)
__global__ void __launch_bounds__(96) mt_hypotheses_b(const int* __restrict__ n_matches, int iters,
                                                      const int* __restrict__ nt,
                                                      const unsigned char* __restrict__ uni,
                                                      const unsigned* __restrict__ rnd,
                                                      const double* __restrict__ xyuv, double* __restrict__ hyp,
                                                      int* __restrict__ valid) {
    __shared__ BlockSolve b;
    __shared__ int sidx[4];
    const int it = blockIdx.x, t = threadIdx.x;
    if (*n_matches < 4) {
        if (t == 0) valid[it] = 0;
        return;
    }
    if (t == 0) {
        const int n = nt[it];
        const unsigned* rw = rnd + 4 * (size_t)it;
        int idx[4];
        if (uni[it]) {
            for (int k = 0; k < 4; ++k) idx[k] = nth_free((int)(rw[k] % (unsigned)(n - k)), idx, k);
        } else {
            idx[0] = n - 1;
            int chosen[3];
            for (int k = 0; k < 3; ++k) {
                chosen[k] = nth_free((int)(rw[k] % (unsigned)(n - 1 - k)), chosen, k);
                idx[k + 1] = chosen[k];
            }
        }
        for (int k = 0; k < 4; ++k) sidx[k] = idx[k];
    }
    __syncthreads();
    if (t < 72) {
        // rows 2k, 2k+1 of pair k: (x, y, 1, 0, 0, 0, -ux, -uy | u), (0, 0, 0, x, y, 1, -vx, -vy | v)
        const int i = t / 9, j = t - 9 * (t / 9), k = i >> 1, m = sidx[k];
        const double x = xyuv[4 * m], y = xyuv[4 * m + 1], u = xyuv[4 * m + 2], v = xyuv[4 * m + 3];
        const double w = (i & 1) ? v : u;
        double e;
        if (j == 8) e = w;
        else if (j == 6) e = -dM(w, x);
        else if (j == 7) e = -dM(w, y);
        else {
            const int jj = (i & 1) ? j - 3 : j;  // position within the row's (x, y, 1) block
            e = jj == 0 ? x : jj == 1 ? y : jj == 2 ? 1.0 : 0.0;
        }
        b.A[i][j] = e;
    }
    __syncthreads();
    const bool ok = solve8_block(b);
    if (t == 0) valid[it] = ok ? 1 : 0;
    if (ok && t < 8) hyp[8 * (size_t)it + t] = b.hs[t];
}

__device__ __forceinline__ double inlier_t2(double inlier_px, const Norm& z) {
    const double tn = dM(inlier_px, z.sb);
    return dM(tn, tn);
}

// one block per hypothesis: its inlier count (-1 when not valid)
__global__ void __launch_bounds__(256) mt_score(const int* __restrict__ n_matches, const double* __restrict__ hyp,
                                                const int* __restrict__ valid, const double* __restrict__ xyuv,
                                                const Norm* __restrict__ norm, double inlier_px,
                                                int* __restrict__ counts) {
    __shared__ int s_c;
    const int t = blockIdx.x;
    if (!valid[t]) {
        if (threadIdx.x == 0) counts[t] = -1;
        return;
    }
    const int nm = *n_matches;
    double h[8];
    for (int k = 0; k < 8; ++k) h[k] = hyp[8 * (size_t)t + k];
    const double t2 = inlier_t2(inlier_px, *norm);
    if (threadIdx.x == 0) s_c = 0;
    __syncthreads();
    int c = 0;
    for (int i = threadIdx.x; i < nm; i += blockDim.x)
        c += inlier(h, xyuv[4 * i], xyuv[4 * i + 1], xyuv[4 * i + 2], xyuv[4 * i + 3], t2);
    for (int off = 16; off > 0; off >>= 1) c += __shfl_down_sync(0xffffffffu, c, off);
    if ((threadIdx.x & 31) == 0) atomicAdd(&s_c, c);
    __syncthreads();
    if (threadIdx.x == 0) counts[t] = s_c;
}

// one block: the best hypothesis (most inliers, ties to the earliest iteration) and its inlier
// flags; best = {iteration or -1, count}
__global__ void __launch_bounds__(256) mt_best(const int* __restrict__ n_matches, int iters,
                                               const double* __restrict__ hyp, const int* __restrict__ counts,
                                               const double* __restrict__ xyuv, const Norm* __restrict__ norm,
                                               double inlier_px, int* __restrict__ best, unsigned char* __restrict__ inl) {
    __shared__ long long s_red[8];
    __shared__ int s_best;
    const int nm = *n_matches, t = threadIdx.x;
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
        // invalid hypotheses (count -1) have key (0 << 32 | .): no model
        const int bt = (b >> 32) > 0 ? (int)(0xffffffffu - (unsigned)(b & 0xffffffffll)) : -1;
        const int bc = (int)(b >> 32) - 1;
        s_best = bt >= 0 && bc >= 4 ? bt : -1;
        best[0] = s_best;
        best[1] = bc;
    }
    __syncthreads();
    const int bt = s_best;
    if (bt < 0) {
        for (int i = t; i < nm; i += blockDim.x) inl[i] = 0;
        return;
    }
    double h[8];
    for (int k = 0; k < 8; ++k) h[k] = hyp[8 * (size_t)bt + k];
    const double t2 = inlier_t2(inlier_px, *norm);
    for (int i = t; i < nm; i += blockDim.x)
        inl[i] = inlier(h, xyuv[4 * i], xyuv[4 * i + 1], xyuv[4 * i + 2], xyuv[4 * i + 3], t2) ? 1 : 0;
}

// the least-squares normal equations on the best hypothesis' inliers: 64 entries of M and 8 of r,
// one warp each.  The two DLT rows of a match are
//   row0 = (x, y, 1, 0, 0, 0, -ux, -uy), row1 = (0, 0, 0, x, y, 1, -vx, -vy),
// M[p][q] += row0[p] row0[q] + row1[p] row1[q], r[p] += row0[p] u + row1[p] v, in quality order.
// The lanes form the products (32 matches at a time, stored in quality order); one lane sums them
// in order.  A product with a structural zero adds +-0 to a sum that is never
// -0, so it is skipped without changing a bit.
__global__ void __launch_bounds__(32) mt_sums(const int* __restrict__ n_matches, const int* __restrict__ best,
                                              const unsigned char* __restrict__ inl, const double* __restrict__ xyuv,
                                              double* __restrict__ sums) {
    if (best[0] < 0) return;
    const int nm = *n_matches, lane = threadIdx.x;
    const int e = blockIdx.x;
    const bool isr = e >= 64;
    const int p = isr ? e - 64 : e / 8, q = isr ? 0 : e % 8;
    const bool p0 = p < 3 || p > 5, p1 = p > 2, q0 = q < 3 || q > 5, q1 = q > 2;
    const bool use0 = isr ? p0 : (p0 && q0), use1 = isr ? p1 : (p1 && q1);
    auto r0 = [](int k, double x, double y, double u) {
        return k == 0 ? x : k == 1 ? y : k == 2 ? 1.0 : k == 6 ? -dM(u, x) : -dM(u, y);
    };
    auto r1 = [](int k, double x, double y, double v) {
        return k == 3 ? x : k == 4 ? y : k == 5 ? 1.0 : k == 6 ? -dM(v, x) : -dM(v, y);
    };
    // the products of every inlier, in quality order, into shared memory
    __shared__ double s0[MT_MAX_POINTS], s1[MT_MAX_POINTS];
    int n = 0;
    for (int i0 = 0; i0 < nm; i0 += 32) {
        const int i = i0 + lane;
        const bool f = i < nm && inl[i];
        const unsigned bal = __ballot_sync(0xffffffffu, f);
        if (f) {
            const double x = xyuv[4 * i], y = xyuv[4 * i + 1], u = xyuv[4 * i + 2], v = xyuv[4 * i + 3];
            const int pos = n + __popc(bal & ((1u << lane) - 1u));
            s0[pos] = use0 ? dM(r0(p, x, y, u), isr ? u : r0(q, x, y, u)) : 0.0;
            s1[pos] = use1 ? dM(r1(p, x, y, v), isr ? v : r1(q, x, y, v)) : 0.0;
        }
        n += __popc(bal);
    }
    __syncwarp();
    if (lane != 0) return;
    double acc = 0.0;
    if (use0 && use1) {
#pragma unroll 8
        for (int j = 0; j < n; ++j) acc = dA(dA(acc, s0[j]), s1[j]);
    } else if (use0) {
#pragma unroll 8
        for (int j = 0; j < n; ++j) acc = dA(acc, s0[j]);
    } else if (use1) {
#pragma unroll 8
        for (int j = 0; j < n; ++j) acc = dA(acc, s1[j]);
    }
    sums[e] = acc;
}

// one block of 96 threads: solve the normal equations (the 4-point hypothesis when singular) and
// go back to pixels, H = Tb^-1 Hn Ta with h33 = 1; identity and 0 inliers when there is no model
__global__ void __launch_bounds__(96) mt_solve(const int* __restrict__ best, const double* __restrict__ hyp,
                                               const double* __restrict__ sums, const Norm* __restrict__ norm,
                                               double* __restrict__ H, int* __restrict__ n_inliers) {
    __shared__ BlockSolve b;
    __shared__ double P[9], Q[9];
    const int t = threadIdx.x, bt = best[0];
    if (bt < 0) {
        if (t < 9) H[t] = t % 4 == 0 ? 1.0 : 0.0;
        if (t == 0) *n_inliers = 0;
        return;
    }
    if (t < 72) {
        const int i = t / 9, j = t - 9 * (t / 9);
        b.A[i][j] = j < 8 ? sums[8 * i + j] : sums[64 + i];
    }
    __syncthreads();
    if (!solve8_block(b)) {
        if (t < 8) b.hs[t] = hyp[8 * (size_t)bt + t];
        __syncthreads();
    }
    const Norm z = *norm;
    // Hn = [h0 h1 h2; h3 h4 h5; h6 h7 1], Ta = [sa 0 -sa ca0; 0 sa -sa ca1; 0 0 1],
    // Tb^-1 = [1/sb 0 cb0; 0 1/sb cb1; 0 0 1]
    if (t < 9) {
        const int r = t / 3, k = t - 3 * (t / 3);
        const double Hn[9] = {b.hs[0], b.hs[1], b.hs[2], b.hs[3], b.hs[4], b.hs[5], b.hs[6], b.hs[7], 1.0};
        const double Ta[9] = {z.sa, 0.0, -dM(z.sa, z.ca0), 0.0, z.sa, -dM(z.sa, z.ca1), 0.0, 0.0, 1.0};
        P[t] = dA(dA(dM(Hn[3 * r], Ta[k]), dM(Hn[3 * r + 1], Ta[3 + k])), dM(Hn[3 * r + 2], Ta[6 + k]));
    }
    __syncthreads();
    if (t < 9) {
        const int r = t / 3, k = t - 3 * (t / 3);
        const double Tbi[9] = {dD(1.0, z.sb), 0.0, z.cb0, 0.0, dD(1.0, z.sb), z.cb1, 0.0, 0.0, 1.0};
        Q[t] = dA(dA(dM(Tbi[3 * r], P[k]), dM(Tbi[3 * r + 1], P[3 + k])), dM(Tbi[3 * r + 2], P[6 + k]));
    }
    __syncthreads();
    if (t < 9) H[t] = dD(Q[t], Q[8]);
    if (t == 0) *n_inliers = best[1];
}

}  // namespace

struct stitch_matcher {
    int device = 0, max_points = 0, max_iters = 0;
    unsigned* keys = nullptr;
    int* ord = nullptr;
    int* dir = nullptr;
    int* best = nullptr;
    Norm* norm = nullptr;
    int* nt = nullptr;
    unsigned char* uni = nullptr;
    double* hyp = nullptr;
    int* valid = nullptr;
    int* counts = nullptr;
    double* xyuv = nullptr;
    int* pick = nullptr;  // best hypothesis: iteration (or -1), inlier count
    double* sums = nullptr;
};

static void matcher_free(stitch_matcher* c) {
    if (!c) return;
    cudaFree(c->keys);
    cudaFree(c->ord);
    cudaFree(c->dir);
    cudaFree(c->best);
    cudaFree(c->norm);
    cudaFree(c->nt);
    cudaFree(c->uni);
    cudaFree(c->hyp);
    cudaFree(c->valid);
    cudaFree(c->counts);
    cudaFree(c->xyuv);
    cudaFree(c->pick);
    cudaFree(c->sums);
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
               cudaMalloc(&c->dir, sizeof(int) * MT_MAX_TABLES * MT_DIR) == cudaSuccess &&
               cudaMalloc(&c->best, sizeof(int) * 2 * max_points) == cudaSuccess &&
               cudaMalloc(&c->norm, sizeof(Norm)) == cudaSuccess && cudaMalloc(&c->nt, sizeof(int) * it) == cudaSuccess &&
               cudaMalloc(&c->uni, it) == cudaSuccess && cudaMalloc(&c->hyp, sizeof(double) * 8 * it) == cudaSuccess &&
               cudaMalloc(&c->valid, sizeof(int) * it) == cudaSuccess &&
               cudaMalloc(&c->counts, sizeof(int) * it) == cudaSuccess &&
               cudaMalloc(&c->xyuv, sizeof(double) * 4 * max_points) == cudaSuccess &&
               cudaMalloc(&c->pick, sizeof(int) * 2) == cudaSuccess && cudaMalloc(&c->sums, sizeof(double) * 72) == cudaSuccess;
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
    mt_build<<<lb.L, 1024, 0, s>>>(db, count_b, lb, c->keys, c->ord, c->dir, cap);
    mt_query<<<(cap + 7) / 8, 256, 0, s>>>(da, count_a, db, count_b, lb, c->keys, c->ord, c->dir, cap,
                                           prm->max_dist, prm->ratio_num, prm->ratio_den, c->best);
    mt_order<<<1, 1024, 0, s>>>(c->best, count_a, cap, xy_a, xy_b, matches, n_matches, c->norm);
    const int iters = prm->iters;
    mt_prep<<<1, 1024, 0, s>>>(n_matches, matches, xy_a, xy_b, c->norm, iters, c->xyuv, c->nt, c->uni);
    if (iters > 0) {
        mt_hypotheses_b<<<iters, 96, 0, s>>>(n_matches, iters, c->nt, c->uni, rnd, c->xyuv, c->hyp, c->valid);
        mt_score<<<iters, 256, 0, s>>>(n_matches, c->hyp, c->valid, c->xyuv, c->norm, prm->inlier_px, c->counts);
    }
    mt_best<<<1, 256, 0, s>>>(n_matches, iters, c->hyp, c->counts, c->xyuv, c->norm, prm->inlier_px, c->pick, inlier);
    mt_sums<<<72, 32, 0, s>>>(n_matches, c->pick, inlier, c->xyuv, c->sums);
    mt_solve<<<1, 96, 0, s>>>(c->pick, c->hyp, c->sums, c->norm, H, n_inliers);
    stitch_status st = cudaGetLastError() == cudaSuccess ? STITCH_OK : STITCH_ECUDA;
    if (prev >= 0 && prev != c->device) cudaSetDevice(prev);
    return st;
}
