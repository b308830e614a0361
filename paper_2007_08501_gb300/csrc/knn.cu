// Exact K nearest neighbours and the Chamfer loss on packed heterogeneous
// point-cloud batches for sm_103a (Section 3.1 of the paper, "3D operators":
// "K Nearest Neighbors" and "Chamfer loss", Eq. 1), with the C ABI of
// include/knn.h.
//
//   k_knn_plan   one block per problem: tiles per cloud (ceil(len1 / queries
//                per block)) and their exclusive prefix, so that one launch
//                covers a heterogeneous batch without a host round trip
//   k_knn<D,KM,QB>  (K <= 4) one block per tile of queries of one cloud: the
//                cloud's candidates pass through shared memory in chunks
//                (pairs of candidates interleaved by coordinate); a group of
//                G consecutive lanes shares QB queries and splits the
//                candidates among its lanes; distances of two candidates at a
//                time in packed f32x2 arithmetic (two lanes of fp32 per
//                instruction, each rounded as plain fp32); register top-K per
//                query (K of KM slots); the group's lists merge through warp
//                shuffles.  Two problems (both directions of a Chamfer loss)
//                can share one launch.
//   k_knn_coop<D,KM,QB>  (K >= 5) the same scan with every lane of a warp on
//                the same candidates for its own queries; the lists live in
//                shared memory and each admitted candidate is inserted by the
//                whole warp (a ballot ranks it, later entries shift a lane)
//   k_pair_sums / k_mean   per-pair Chamfer terms and the batch mean, fixed
//                reduction order
//   k_chamfer_bwd / k_knn_bwd   gradients, scatter to the neighbours with
//                warp aggregation by target row
#include <cuda_runtime.h>

#include <climits>
#include <cstdint>

#include "knn.h"
#include "meshrast.h"
#include "rast_common.cuh"

namespace mr {
namespace {

constexpr int kThreads = 256;
constexpr int kChunk = 2048;   // candidates per shared-memory chunk (even)

struct KnnProblem {
    const float *p1, *p2;
    const int64_t *first1, *len1, *first2;
    const int64_t *len2;
    int64_t *idx;
    float *dists;
    long long *tiles;   // (N + 1): exclusive prefix of tiles per cloud, tiles[N] = total
    int N, K, G, qpb;   // qpb: queries per block = (kThreads / G) * QB
    int block0;         // first block of this problem in the launch
};

struct KnnArgs {
    KnnProblem pr[2];
    int nprob;
};

// ---------------------------------------------------------------------------
// plan: tiles of each cloud and their exclusive prefix (one block per problem)
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(1024) k_knn_plan(KnnArgs a) {
    const KnnProblem &P = a.pr[blockIdx.x];
    __shared__ long long s_warp[32];
    __shared__ long long s_carry;
    if (threadIdx.x == 0) s_carry = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int base = 0; base < P.N; base += 1024) {
        const int i = base + threadIdx.x;
        long long v = 0;
        if (i < P.N) {
            const long long n = P.len1[i];
            v = n > 0 ? (n + P.qpb - 1) / P.qpb : 0;
        }
        long long x = v;   // inclusive scan within the warp
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const long long y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) s_warp[w] = x;
        __syncthreads();
        if (w == 0) {
            long long t = s_warp[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const long long y = __shfl_up_sync(0xffffffffu, t, o);
                if (lane >= o) t += y;
            }
            s_warp[lane] = t;   // inclusive over warps
        }
        __syncthreads();
        const long long carry = s_carry;
        const long long before = carry + (w > 0 ? s_warp[w - 1] : 0) + x - v;
        if (i < P.N) P.tiles[i] = before;
        __syncthreads();
        if (threadIdx.x == 0) s_carry = carry + s_warp[31];
        __syncthreads();
    }
    if (threadIdx.x == 0) P.tiles[P.N] = s_carry;
}

// ---------------------------------------------------------------------------
// packed two-lane fp32 arithmetic (each lane rounded to nearest even, no ftz)
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long f2_dup(float x) {
    unsigned long long r;
    asm("mov.b64 %0, {%1, %1};" : "=l"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ unsigned long long f2_sub(unsigned long long a, unsigned long long b) {
    unsigned long long r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ unsigned long long f2_mul(unsigned long long a, unsigned long long b) {
    unsigned long long r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ unsigned long long f2_fma(unsigned long long a, unsigned long long b,
                                                     unsigned long long c) {
    unsigned long long r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}
__device__ __forceinline__ void f2_split(unsigned long long v, float &lo, float &hi) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}

// ranking key: ascending distance, then ascending candidate row
__device__ __forceinline__ bool nn_before(float d, int j, float e, int k) { return d < e || (d == e && j < k); }

// the K best (distance, local row) pairs so far, ascending, right-aligned in
// KM slots: slots below KM - K hold -inf and never move, so the K-th best --
// the admission threshold and the entry a new one evicts -- is always slot
// KM - 1 (no register array is ever indexed by a run-time value)
template <int KM>
struct NnList {
    float z[KM];
    int f[KM];
    __device__ __forceinline__ void init(int K) {
#pragma unroll
        for (int k = 0; k < KM; ++k) {
            z[k] = k < KM - K ? __int_as_float(0xff800000) : __int_as_float(0x7f800000);
            f[k] = INT_MAX;
        }
    }
    // insertion during the scan: a thread meets its candidates in increasing
    // row order, so a new entry goes after the entries of equal distance and
    // the distance alone decides
    __device__ __forceinline__ void push(float d, int j) {
        z[KM - 1] = d;
        f[KM - 1] = j;
#pragma unroll
        for (int k = KM - 1; k > 0; --k) {
            const bool sw = z[k] < z[k - 1];
            const float tz = z[k - 1];
            const int tf = f[k - 1];
            z[k - 1] = sw ? z[k] : tz;
            f[k - 1] = sw ? f[k] : tf;
            z[k] = sw ? tz : z[k];
            f[k] = sw ? tf : f[k];
        }
    }
    // insertion of another lane's entry (full ranking key)
    __device__ __forceinline__ void insert(float d, int j) {
        z[KM - 1] = d;
        f[KM - 1] = j;
#pragma unroll
        for (int k = KM - 1; k > 0; --k) {
            const bool sw = nn_before(z[k], f[k], z[k - 1], f[k - 1]);
            const float tz = z[k - 1];
            const int tf = f[k - 1];
            z[k - 1] = sw ? z[k] : tz;
            f[k - 1] = sw ? f[k] : tf;
            z[k] = sw ? tz : z[k];
            f[k] = sw ? tf : f[k];
        }
    }
};

// chunk layout: candidates 2p and 2p + 1 form pair p; SA[p] = (x, x', y, y'),
// SB[p] = (z, z', w, w'), so one 16-byte load gives two coordinates of both
template <int D>
struct PairCoords {
    unsigned long long c[D];
};

template <int D>
__device__ __forceinline__ PairCoords<D> load_pair(const float4 *SA, const float4 *SB, int p) {
    PairCoords<D> r;
    if (D >= 2) {
        const ulonglong2 a = *reinterpret_cast<const ulonglong2 *>(SA + p);
        r.c[0] = a.x;
        r.c[D >= 2 ? 1 : 0] = a.y;
    } else {
        r.c[0] = *reinterpret_cast<const unsigned long long *>(SA + p);
    }
    if (D == 4) {
        const ulonglong2 b = *reinterpret_cast<const ulonglong2 *>(SB + p);
        r.c[D >= 3 ? 2 : 0] = b.x;
        r.c[D >= 4 ? 3 : 0] = b.y;
    } else if (D == 3) {
        r.c[D >= 3 ? 2 : 0] = *reinterpret_cast<const unsigned long long *>(SB + p);
    }
    return r;
}

// squared distances of one query (coordinates duplicated in both lanes) to a pair
template <int D>
__device__ __forceinline__ void pair_dist(const unsigned long long (&q)[D], const PairCoords<D> &X, float &s0,
                                          float &s1) {
    unsigned long long dx = f2_sub(q[0], X.c[0]);
    unsigned long long s = f2_mul(dx, dx);
#pragma unroll
    for (int c = 1; c < D; ++c) {
        dx = f2_sub(q[c], X.c[c]);
        s = f2_fma(dx, dx, s);
    }
    f2_split(s, s0, s1);
}

template <int KM>
__device__ __forceinline__ void take1(NnList<KM> &L, float &thr, float d, int j) {
    const bool lt = d < thr;
    thr = lt ? d : thr;
    L.z[0] = lt ? d : L.z[0];
    L.f[0] = lt ? j : L.f[0];
}

template <int D, int KM, int QB>
__global__ void __launch_bounds__(kThreads, KM <= 2 ? 4 : 3) k_knn(KnnArgs a) {
    const int pb = (a.nprob > 1 && (int)blockIdx.x >= a.pr[1].block0) ? 1 : 0;
    const KnnProblem &P = a.pr[pb];
    const long long b = (long long)blockIdx.x - P.block0;
    const long long total = P.tiles[P.N];
    if (b >= total) return;   // uniform for the block, before any barrier
    // cloud of this tile: the last i with tiles[i] <= b (tiles[0] = 0 <= b < tiles[N])
    int lo = 0, hi = P.N;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (P.tiles[mid] <= b) lo = mid; else hi = mid;
    }
    const int ci = lo;
    const long long t = b - P.tiles[ci];
    const int G = P.G, K = P.K;
    const int grp = threadIdx.x / G, gl = threadIdx.x - grp * G;
    const long long qbase = P.first1[ci] + t * P.qpb;
    const long long qend = P.first1[ci] + P.len1[ci];
    const long long c0 = P.first2[ci];
    const int cn = (int)P.len2[ci];

    unsigned long long qq[QB][D];   // each query coordinate duplicated in both lanes
    bool valid[QB];
    long long row[QB];
#pragma unroll
    for (int u = 0; u < QB; ++u) {
        row[u] = qbase + (long long)grp * QB + u;
        valid[u] = row[u] < qend;
#pragma unroll
        for (int c = 0; c < D; ++c) qq[u][c] = f2_dup(valid[u] ? P.p1[row[u] * D + c] : 0.f);
    }
    NnList<KM> L[QB];
    float thr[QB];
#pragma unroll
    for (int u = 0; u < QB; ++u) {
        L[u].init(K);
        thr[u] = __int_as_float(0x7f800000);
    }

    __shared__ __align__(16) float4 SA[kChunk / 2 + 1];
    __shared__ __align__(16) float4 SB[D > 2 ? kChunk / 2 + 1 : 1];
    for (int base = 0; base < cn; base += kChunk) {
        const int cnt = min(kChunk, cn - base);
        __syncthreads();   // the previous chunk is consumed
        const float *src = P.p2 + (c0 + base) * D;
        const int npair = (cnt + 1) >> 1;
        // one thread per pair: 2 D coalesced loads, one 16-byte (and one 8- or
        // 16-byte) shared store; an odd last slot gets x = +inf (never admitted)
#pragma unroll 1
        for (int pp = threadIdx.x; pp < npair; pp += kThreads) {
            float v0[4] = {0.f, 0.f, 0.f, 0.f}, v1[4] = {0.f, 0.f, 0.f, 0.f};
            const bool two = 2 * pp + 1 < cnt;
#pragma unroll
            for (int c = 0; c < D; ++c) {
                v0[c] = src[2 * pp * D + c];
                v1[c] = two ? src[(2 * pp + 1) * D + c] : (c == 0 ? __int_as_float(0x7f800000) : 0.f);
            }
            SA[pp] = make_float4(v0[0], v1[0], v0[1], v1[1]);
            if (D > 2) SB[pp] = make_float4(v0[2], v1[2], v0[3], v1[3]);
        }
        __syncthreads();
        int jp = gl;
        // two pairs per step: one admission test per query for four candidates
        for (; jp + G < npair; jp += 2 * G) {
            const PairCoords<D> X = load_pair<D>(SA, SB, jp);
            const PairCoords<D> Y = load_pair<D>(SA, SB, jp + G);
#pragma unroll
            for (int u = 0; u < QB; ++u) {
                float s0, s1, t0, t1;
                pair_dist<D>(qq[u], X, s0, s1);
                pair_dist<D>(qq[u], Y, t0, t1);
                if (fminf(fminf(s0, s1), fminf(t0, t1)) < thr[u]) {
                    const int ja = base + 2 * jp, jb = base + 2 * (jp + G);
                    if (KM == 1) {   // predicated, in row order
                        take1(L[u], thr[u], s0, ja);
                        take1(L[u], thr[u], s1, ja + 1);
                        take1(L[u], thr[u], t0, jb);
                        take1(L[u], thr[u], t1, jb + 1);
                    } else {
                        // in row order; one insertion site per query keeps the
                        // unrolled list in registers
#pragma unroll 1
                        for (int h = 0; h < 4; ++h) {
                            const float d = h == 0 ? s0 : (h == 1 ? s1 : (h == 2 ? t0 : t1));
                            if (d < thr[u]) {
                                L[u].push(d, (h < 2 ? ja : jb) + (h & 1));
                                thr[u] = L[u].z[KM - 1];
                            }
                        }
                    }
                }
            }
        }
        if (jp < npair) {
            const PairCoords<D> X = load_pair<D>(SA, SB, jp);
#pragma unroll
            for (int u = 0; u < QB; ++u) {
                float s0, s1;
                pair_dist<D>(qq[u], X, s0, s1);
                if (s0 < thr[u]) {
                    L[u].push(s0, base + 2 * jp);
                    thr[u] = L[u].z[KM - 1];
                }
                if (s1 < thr[u]) {
                    L[u].push(s1, base + 2 * jp + 1);
                    thr[u] = L[u].z[KM - 1];
                }
            }
        }
    }

    // merge the group's lists: lane gl pulls the list of lane gl + o
    for (int o = 1; o < G; o <<= 1) {
        const bool recv = (gl & (2 * o - 1)) == 0;
#pragma unroll
        for (int u = 0; u < QB; ++u) {
#pragma unroll
            for (int k = 0; k < KM; ++k) {
                const float v = __shfl_down_sync(0xffffffffu, L[u].z[k], o);
                const int w = __shfl_down_sync(0xffffffffu, L[u].f[k], o);
                if (recv && k >= KM - K && nn_before(v, w, L[u].z[KM - 1], L[u].f[KM - 1])) L[u].insert(v, w);
            }
        }
    }
    if (gl != 0) return;
#pragma unroll
    for (int u = 0; u < QB; ++u) {
        if (!valid[u]) continue;
#pragma unroll
        for (int k = 0; k < KM; ++k) {
            const int r = k - (KM - K);   // rank of slot k
            if (r < 0) continue;
            const bool has = L[u].f[k] != INT_MAX;
            P.idx[row[u] * K + r] = has ? c0 + L[u].f[k] : -1;
            P.dists[row[u] * K + r] = has ? L[u].z[k] : __int_as_float(0x7f800000);
        }
    }
}

// ---------------------------------------------------------------------------
// K >= 5: QB queries per lane (2, or 1 for K > 8), every lane of a warp
// scanning the same candidates; an admitted candidate is inserted by the whole warp into its
// query's list in shared memory (lane k holds entry k; the lanes before the
// new key keep theirs, the others shift by one), one admission at a time, so
// that no lane idles through another lane's K-step insertion.  Keys pack the
// fp32 distance bits (non-negative, so ordered as integers) above the local
// candidate row: comparing keys is the (distance, row) ranking.
// ---------------------------------------------------------------------------
constexpr unsigned long long kEmptyKey = 0x7f800000ffffffffull;   // (+inf, no row)

template <int KM>
__device__ __forceinline__ void coop_admit(unsigned long long *W, unsigned pend, const float (&c)[4], int j0, int K,
                                           float &thr) {
    const int lane = threadIdx.x & 31;
    while (pend) {
        const int src = __ffs(pend) - 1;
        pend &= pend - 1;
        float th = __shfl_sync(0xffffffffu, thr, src);
        unsigned long long *Lq = W + src * KM;
#pragma unroll
        for (int h = 0; h < 4; ++h) {
            const float d = __shfl_sync(0xffffffffu, c[h], src);
            if (!(d < th)) continue;   // uniform: d and th are the source lane's
            const unsigned long long key = ((unsigned long long)__float_as_uint(d) << 32) | (unsigned)(j0 + h);
            const unsigned long long e = lane < K ? Lq[lane] : kEmptyKey;
            const int pos = __popc(__ballot_sync(0xffffffffu, lane < K && e < key));
            const unsigned long long prev = __shfl_up_sync(0xffffffffu, e, 1);
            const unsigned long long ne = lane < pos ? e : (lane == pos ? key : prev);
            if (lane < K) Lq[lane] = ne;
            th = __uint_as_float((unsigned)(__shfl_sync(0xffffffffu, ne, K - 1) >> 32));
            __syncwarp();
        }
        if (lane == src) thr = th;
    }
}

template <int D, int KM, int QB>
__global__ void __launch_bounds__(kThreads, KM <= 16 ? 3 : 2) k_knn_coop(KnnArgs a) {
    const int pb = (a.nprob > 1 && (int)blockIdx.x >= a.pr[1].block0) ? 1 : 0;
    const KnnProblem &P = a.pr[pb];
    const long long b = (long long)blockIdx.x - P.block0;
    const long long total = P.tiles[P.N];
    if (b >= total) return;   // uniform for the block, before any barrier
    int lo = 0, hi = P.N;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (P.tiles[mid] <= b) lo = mid; else hi = mid;
    }
    const int ci = lo;
    const long long t = b - P.tiles[ci];
    const int K = P.K;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const long long qend = P.first1[ci] + P.len1[ci];
    const long long c0 = P.first2[ci];
    const int cn = (int)P.len2[ci];
    // QB queries per lane: query u of the block's tile is row base + u * 256 + thread
    unsigned long long qq[QB][D];
    long long row[QB];
    bool valid[QB];
    float thr[QB];
#pragma unroll
    for (int u = 0; u < QB; ++u) {
        row[u] = P.first1[ci] + t * P.qpb + u * kThreads + threadIdx.x;
        valid[u] = row[u] < qend;
#pragma unroll
        for (int c = 0; c < D; ++c) qq[u][c] = f2_dup(valid[u] ? P.p1[row[u] * D + c] : 0.f);
        // a lane without a query admits nothing
        thr[u] = valid[u] ? __int_as_float(0x7f800000) : __int_as_float(0xff800000);
    }

    extern __shared__ unsigned long long s_lists[];   // [warp][u][query lane][KM]
    unsigned long long *W = s_lists + (size_t)warp * QB * 32 * KM;
    for (int e = lane; e < QB * 32 * KM; e += 32) W[e] = kEmptyKey;
    __syncwarp();

    __shared__ __align__(16) float4 SA[kChunk / 2 + 1];
    __shared__ __align__(16) float4 SB[D > 2 ? kChunk / 2 + 1 : 1];
    for (int base = 0; base < cn; base += kChunk) {
        const int cnt = min(kChunk, cn - base);
        __syncthreads();   // the previous chunk is consumed
        const float *src = P.p2 + (c0 + base) * D;
        const int npair = (cnt + 1) >> 1;
#pragma unroll 1
        for (int pp = threadIdx.x; pp < npair; pp += kThreads) {
            float v0[4] = {0.f, 0.f, 0.f, 0.f}, v1[4] = {0.f, 0.f, 0.f, 0.f};
            const bool two = 2 * pp + 1 < cnt;
#pragma unroll
            for (int c = 0; c < D; ++c) {
                v0[c] = src[2 * pp * D + c];
                v1[c] = two ? src[(2 * pp + 1) * D + c] : (c == 0 ? __int_as_float(0x7f800000) : 0.f);
            }
            SA[pp] = make_float4(v0[0], v1[0], v0[1], v1[1]);
            if (D > 2) SB[pp] = make_float4(v0[2], v1[2], v0[3], v1[3]);
        }
        __syncthreads();
        int jp = 0;
        for (; jp + 1 < npair; jp += 2) {   // uniform: every lane takes the same candidates
            const PairCoords<D> X = load_pair<D>(SA, SB, jp);
            const PairCoords<D> Y = load_pair<D>(SA, SB, jp + 1);
#pragma unroll
            for (int u = 0; u < QB; ++u) {
                float c[4];
                pair_dist<D>(qq[u], X, c[0], c[1]);
                pair_dist<D>(qq[u], Y, c[2], c[3]);
                const unsigned pend =
                    __ballot_sync(0xffffffffu, fminf(fminf(c[0], c[1]), fminf(c[2], c[3])) < thr[u]);
                if (pend) coop_admit<KM>(W + u * 32 * KM, pend, c, base + 2 * jp, K, thr[u]);
            }
        }
        if (jp < npair) {
            const PairCoords<D> X = load_pair<D>(SA, SB, jp);
#pragma unroll
            for (int u = 0; u < QB; ++u) {
                float c[4];
                pair_dist<D>(qq[u], X, c[0], c[1]);
                c[2] = c[3] = __int_as_float(0x7f800000);
                const unsigned pend = __ballot_sync(0xffffffffu, fminf(c[0], c[1]) < thr[u]);
                if (pend) coop_admit<KM>(W + u * 32 * KM, pend, c, base + 2 * jp, K, thr[u]);
            }
        }
    }
    __syncwarp();
#pragma unroll
    for (int u = 0; u < QB; ++u) {
        if (!valid[u]) continue;
        const unsigned long long *Lq = W + (u * 32 + lane) * KM;
        for (int k = 0; k < K; ++k) {
            const unsigned long long key = Lq[k];
            const bool has = key != kEmptyKey;
            P.idx[row[u] * K + k] = has ? c0 + (long long)(unsigned)(key & 0xffffffffull) : -1;
            P.dists[row[u] * K + k] = has ? __uint_as_float((unsigned)(key >> 32)) : __int_as_float(0x7f800000);
        }
    }
}

// ---------------------------------------------------------------------------
// Chamfer reductions: per pair, then the batch mean (fixed order)
// ---------------------------------------------------------------------------
// sum over the block in a fixed order (shuffle tree per warp, then over warps); result in thread 0
__device__ __forceinline__ double block_sum(double v, double *s_red) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) s_red[w] = v;
    __syncthreads();
    double r = 0.0;
    if (w == 0) {
        r = lane < (int)(blockDim.x >> 5) ? s_red[lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) r += __shfl_down_sync(0xffffffffu, r, o);
    }
    return r;
}

struct PairArgs {
    const int64_t *first1, *len1, *first2, *len2;
    const int64_t *idx_pq, *idx_qp;
    const float *d_pq, *d_qp;
    float *per_pair, *loss;
    int N;
};

// FP64 accumulation: a few adds per thread, far from any throughput limit
__global__ void __launch_bounds__(256) k_pair_sums(PairArgs a) {
    __shared__ double s_red[32];
    const int i = blockIdx.x;
    double out = 0.0;
    for (int dir = 0; dir < 2; ++dir) {
        const int64_t f = dir ? a.first2[i] : a.first1[i];
        const int64_t n = dir ? a.len2[i] : a.len1[i];
        const int64_t *ix = dir ? a.idx_qp : a.idx_pq;
        const float *d = dir ? a.d_qp : a.d_pq;
        double s = 0.0;
        for (int64_t r = f + threadIdx.x; r < f + n; r += blockDim.x)
            if (ix[r] >= 0) s += d[r];
        s = block_sum(s, s_red);
        if (threadIdx.x == 0 && n > 0) out += s / (double)n;
    }
    if (threadIdx.x == 0) a.per_pair[i] = (float)out;
}

__global__ void __launch_bounds__(1024) k_mean(PairArgs a) {
    __shared__ double s_red[32];
    double s = 0.0;
    for (int i = threadIdx.x; i < a.N; i += blockDim.x) s += a.per_pair[i];
    s = block_sum(s, s_red);
    if (threadIdx.x == 0) a.loss[0] = a.N > 0 ? (float)(s / a.N) : 0.f;
}

// ---------------------------------------------------------------------------
// gradients
// ---------------------------------------------------------------------------
// the cloud holding packed row r: the last i with first[i] <= r, if r < first[i] + len[i]
__device__ __forceinline__ int cloud_of(long long r, const int64_t *first, const int64_t *len, int N) {
    int lo = 0, hi = N;   // answer in [lo, hi)
    if (N == 0 || first[0] > r) return -1;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (first[mid] <= r) lo = mid; else hi = mid;
    }
    return r < first[lo] + len[lo] ? lo : -1;
}

// atomically add -v to grad[target], lanes with equal targets summed first
template <int D>
__device__ __forceinline__ void scatter_neg(long long target, float (&v)[D], float *grad) {
    const unsigned lane = threadIdx.x & 31u;
    const long long key = target >= 0 ? target : -1 - (long long)lane;   // invalid lanes stay alone
    const unsigned peers = __match_any_sync(0xffffffffu, key);
    group_sum<D>(peers, v);
    if (target >= 0 && (__ffs(peers) - 1) == (int)lane) {
#pragma unroll
        for (int c = 0; c < D; ++c) atomicAdd(grad + target * D + c, -v[c]);
    }
}

struct ChamferBwdArgs {
    const float *p, *q;
    const int64_t *first1, *len1, *first2, *len2;
    const int64_t *idx_pq, *idx_qp;
    const float *grad_loss, *grad_per_pair;
    float *grad_p, *grad_q;
    long long P1, P2;
    int N;
};

template <int D>
__global__ void __launch_bounds__(256) k_chamfer_bwd(ChamferBwdArgs a) {
    const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const bool dir = r >= a.P1;   // false: rows of p (p -> q), true: rows of q (q -> p)
    const long long rr = dir ? r - a.P1 : r;
    const bool in_range = r < a.P1 + a.P2;
    const float *x = dir ? a.q : a.p, *y = dir ? a.p : a.q;
    float *gx = dir ? a.grad_q : a.grad_p, *gy = dir ? a.grad_p : a.grad_q;
    long long target = -1;
    float v[D];
#pragma unroll
    for (int c = 0; c < D; ++c) v[c] = 0.f;
    if (in_range) {
        const int i = dir ? cloud_of(rr, a.first2, a.len2, a.N) : cloud_of(rr, a.first1, a.len1, a.N);
        const long long nb = (dir ? a.idx_qp : a.idx_pq)[rr];
        if (i >= 0 && nb >= 0) {
            float w = a.grad_per_pair ? a.grad_per_pair[i] : 0.f;
            if (a.grad_loss) w += a.grad_loss[0] / (float)a.N;
            const float coef = 2.f * w / (float)(dir ? a.len2[i] : a.len1[i]);
#pragma unroll
            for (int c = 0; c < D; ++c) {
                v[c] = coef * (x[rr * D + c] - y[nb * D + c]);
                atomicAdd(gx + rr * D + c, v[c]);
            }
            target = nb;
        }
    }
    // lanes of one warp may straddle the two directions: scatter each separately
    const unsigned both = __ballot_sync(0xffffffffu, dir);
    if (both == 0u || both == 0xffffffffu) {
        scatter_neg<D>(target, v, gy);
    } else {
        float w0[D], w1[D];
#pragma unroll
        for (int c = 0; c < D; ++c) { w0[c] = dir ? 0.f : v[c]; w1[c] = dir ? v[c] : 0.f; }
        scatter_neg<D>(dir ? -1 : target, w0, a.grad_q);
        scatter_neg<D>(dir ? target : -1, w1, a.grad_p);
    }
}

struct KnnBwdArgs {
    const float *p1, *p2;
    const int64_t *idx;
    const float *grad_dists;
    float *grad_p1, *grad_p2;
    long long P1, P2;
    int K;
};

template <int D>
__global__ void __launch_bounds__(256) k_knn_bwd(KnnBwdArgs a) {
    const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const bool in_range = r < a.P1;
    float x[D], own[D];
#pragma unroll
    for (int c = 0; c < D; ++c) {
        x[c] = in_range ? a.p1[r * D + c] : 0.f;
        own[c] = 0.f;
    }
    for (int k = 0; k < a.K; ++k) {
        long long nb = in_range ? a.idx[r * a.K + k] : -1;
        if (nb >= a.P2) nb = -1;
        float v[D];
        if (nb >= 0) {
            const float g2 = 2.f * a.grad_dists[r * a.K + k];
#pragma unroll
            for (int c = 0; c < D; ++c) {
                v[c] = g2 * (x[c] - a.p2[nb * D + c]);
                own[c] += v[c];
            }
        } else {
#pragma unroll
            for (int c = 0; c < D; ++c) v[c] = 0.f;
        }
        scatter_neg<D>(nb, v, a.grad_p2);
    }
    if (in_range) {
#pragma unroll
        for (int c = 0; c < D; ++c) a.grad_p1[r * D + c] = own[c];
    }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
int km_for_knn(int K) {
    int km = 1;
    while (km < K) km <<= 1;
    return km;
}
int qb_for(int km) { return km <= 2 ? 4 : (km <= 8 ? 2 : 1); }
bool coop_for(int km) { return km >= 8; }   // K >= 5: warp-cooperative insertion into shared-memory lists

// lanes per query group: enough threads to fill the GPU twice over, but at
// least 256 candidates per lane on average
int group_for(long long P1, long long P2, long long N, int qb) {
    const long long want = 2LL * 152 * 2048;
    const long long per_cloud = N > 0 ? P2 / N : 0;
    int G = 1;
    while (G < 32 && (P1 * G) / qb < want && per_cloud / (2 * G) >= 256) G <<= 1;
    return G;
}

template <int D, int KM>
cudaError_t launch_knn_coop(const KnnArgs &a, int blocks, cudaStream_t st) {
    constexpr int QB = KM <= 8 ? 2 : 1;
    auto kern = k_knn_coop<D, KM, QB>;
    const int dyn = QB * kThreads * KM * (int)sizeof(unsigned long long);
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn);
    cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
    kern<<<blocks, kThreads, dyn, st>>>(a);
    return cudaGetLastError();
}

template <int D, int KM>
cudaError_t launch_knn_t(const KnnArgs &a, int blocks, cudaStream_t st) {
    constexpr int QB = KM <= 2 ? 4 : (KM <= 4 ? 2 : 1);
    auto kern = k_knn<D, KM, QB>;
    // shared memory for four 33 KB blocks per SM
    cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
    kern<<<blocks, kThreads, 0, st>>>(a);
    return cudaGetLastError();
}

template <int D>
cudaError_t launch_knn_d(const KnnArgs &a, int km, int blocks, cudaStream_t st) {
    switch (km) {
        case 1: return launch_knn_t<D, 1>(a, blocks, st);
        case 2: return launch_knn_t<D, 2>(a, blocks, st);
        case 4: return launch_knn_t<D, 4>(a, blocks, st);
        case 8: return launch_knn_coop<D, 8>(a, blocks, st);
        case 16: return launch_knn_coop<D, 16>(a, blocks, st);
        default: return launch_knn_coop<D, 32>(a, blocks, st);
    }
}

cudaError_t launch_knn(const KnnArgs &a, int D, int km, int blocks, cudaStream_t st) {
    switch (D) {
        case 1: return launch_knn_d<1>(a, km, blocks, st);
        case 2: return launch_knn_d<2>(a, km, blocks, st);
        case 3: return launch_knn_d<3>(a, km, blocks, st);
        default: return launch_knn_d<4>(a, km, blocks, st);
    }
}

size_t ws_bytes(int64_t N) { return (size_t)((2 * (N + 1) * 8 + 255) / 256 * 256); }

bool ws_ok(void *ws, size_t bytes, int64_t N) {
    return ws && (reinterpret_cast<uintptr_t>(ws) & 255u) == 0 && bytes >= ws_bytes(N);
}

// fill one problem; returns its number of blocks (an upper bound of its tiles)
long long set_problem(KnnProblem &pr, const float *p1, int64_t P1, const int64_t *first1, const int64_t *len1,
                      const float *p2, int64_t P2, const int64_t *first2, const int64_t *len2, int64_t N, int K,
                      int km, int64_t *idx, float *dists, long long *tiles, int block0) {
    const int qb = qb_for(km);
    pr.p1 = p1;
    pr.p2 = p2;
    pr.first1 = first1;
    pr.len1 = len1;
    pr.first2 = first2;
    pr.len2 = len2;
    pr.idx = idx;
    pr.dists = dists;
    pr.tiles = tiles;
    pr.N = (int)N;
    pr.K = K;
    pr.G = coop_for(km) ? 1 : group_for(P1, P2, N, qb);
    pr.qpb = kThreads / pr.G * qb;
    pr.block0 = block0;
    return (P1 + pr.qpb - 1) / pr.qpb + N;
}

}  // namespace
}  // namespace mr

using namespace mr;

extern "C" {

MESHRAST_API size_t knn_workspace_bytes(int64_t N) { return N < 0 ? 0 : ws_bytes(N); }

MESHRAST_API int knn_points(const float *p1, int64_t P1, const int64_t *first1, const int64_t *len1,
                            const float *p2, int64_t P2, const int64_t *first2, const int64_t *len2, int64_t N,
                            int32_t D, int32_t K, int64_t *idx, float *dists, void *workspace,
                            size_t workspace_bytes, void *stream) {
    if (N < 0 || N > INT_MAX - 1 || P1 < 0 || P2 < 0 || D < 1 || D > 4 || K < 1 || K > 32)
        return MESHRAST_ERR_INVALID_ARG;
    if (N > 0 && (!first1 || !len1 || !first2 || !len2)) return MESHRAST_ERR_INVALID_ARG;
    if ((P1 > 0 && (!p1 || !idx || !dists)) || (P2 > 0 && !p2)) return MESHRAST_ERR_INVALID_ARG;
    if (!ws_ok(workspace, workspace_bytes, N)) return MESHRAST_ERR_WORKSPACE;
    if (N == 0 || P1 == 0) return MESHRAST_OK;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const int km = km_for_knn(K);
    KnnArgs a{};
    a.nprob = 1;
    const long long blocks = set_problem(a.pr[0], p1, P1, first1, len1, p2, P2, first2, len2, N, K, km, idx, dists,
                                         reinterpret_cast<long long *>(workspace), 0);
    if (blocks > INT_MAX) return MESHRAST_ERR_INVALID_ARG;
    a.pr[1] = a.pr[0];
    k_knn_plan<<<1, 1024, 0, st>>>(a);
    if (cudaGetLastError() != cudaSuccess) return MESHRAST_ERR_CUDA;
    return launch_knn(a, D, km, (int)blocks, st) == cudaSuccess ? MESHRAST_OK : MESHRAST_ERR_CUDA;
}

MESHRAST_API int knn_points_bwd(const float *p1, int64_t P1, const float *p2, int64_t P2, int32_t D, int32_t K,
                                const int64_t *idx, const float *grad_dists, float *grad_p1, float *grad_p2,
                                void *stream) {
    if (P1 < 0 || P2 < 0 || D < 1 || D > 4 || K < 1 || K > 32) return MESHRAST_ERR_INVALID_ARG;
    if ((P1 > 0 && (!p1 || !idx || !grad_dists || !grad_p1)) || (P2 > 0 && (!p2 || !grad_p2)))
        return MESHRAST_ERR_INVALID_ARG;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (P2 > 0 && cudaMemsetAsync(grad_p2, 0, (size_t)P2 * D * sizeof(float), st) != cudaSuccess)
        return MESHRAST_ERR_CUDA;
    if (P1 == 0) return MESHRAST_OK;
    KnnBwdArgs a{p1, p2, idx, grad_dists, grad_p1, grad_p2, P1, P2, K};
    const long long blocks = (P1 + 255) / 256;
    if (blocks > INT_MAX) return MESHRAST_ERR_INVALID_ARG;
    switch (D) {
        case 1: k_knn_bwd<1><<<(int)blocks, 256, 0, st>>>(a); break;
        case 2: k_knn_bwd<2><<<(int)blocks, 256, 0, st>>>(a); break;
        case 3: k_knn_bwd<3><<<(int)blocks, 256, 0, st>>>(a); break;
        default: k_knn_bwd<4><<<(int)blocks, 256, 0, st>>>(a); break;
    }
    return cudaGetLastError() == cudaSuccess ? MESHRAST_OK : MESHRAST_ERR_CUDA;
}

MESHRAST_API int chamfer_fwd(const float *p, int64_t P1, const int64_t *first1, const int64_t *len1,
                             const float *q, int64_t P2, const int64_t *first2, const int64_t *len2, int64_t N,
                             int32_t D, int64_t *idx_pq, float *d_pq, int64_t *idx_qp, float *d_qp,
                             float *loss_per_pair, float *loss, void *workspace, size_t workspace_bytes,
                             void *stream) {
    if (N < 0 || N > INT_MAX - 1 || P1 < 0 || P2 < 0 || D < 1 || D > 4 || !loss) return MESHRAST_ERR_INVALID_ARG;
    if (N > 0 && (!first1 || !len1 || !first2 || !len2 || !loss_per_pair)) return MESHRAST_ERR_INVALID_ARG;
    if ((P1 > 0 && (!p || !idx_pq || !d_pq)) || (P2 > 0 && (!q || !idx_qp || !d_qp))) return MESHRAST_ERR_INVALID_ARG;
    if (!ws_ok(workspace, workspace_bytes, N)) return MESHRAST_ERR_WORKSPACE;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    PairArgs pa{first1, len1, first2, len2, idx_pq, idx_qp, d_pq, d_qp, loss_per_pair, loss, (int)N};
    if (N == 0) {
        k_mean<<<1, 1024, 0, st>>>(pa);
        return cudaGetLastError() == cudaSuccess ? MESHRAST_OK : MESHRAST_ERR_CUDA;
    }
    long long *tiles = reinterpret_cast<long long *>(workspace);
    KnnArgs a{};
    a.nprob = 2;
    // both directions in one launch: blocks [0, b0) find neighbours of p in q, [b0, b0 + b1) of q in p
    const long long b0 = set_problem(a.pr[0], p, P1, first1, len1, q, P2, first2, len2, N, 1, 1, idx_pq, d_pq,
                                     tiles, 0);
    if (b0 > INT_MAX) return MESHRAST_ERR_INVALID_ARG;
    const long long b1 = set_problem(a.pr[1], q, P2, first2, len2, p, P1, first1, len1, N, 1, 1, idx_qp, d_qp,
                                     tiles + (N + 1), (int)b0);
    if (b0 + b1 > INT_MAX) return MESHRAST_ERR_INVALID_ARG;
    k_knn_plan<<<2, 1024, 0, st>>>(a);
    if (cudaGetLastError() != cudaSuccess) return MESHRAST_ERR_CUDA;
    if (launch_knn(a, D, 1, (int)(b0 + b1), st) != cudaSuccess) return MESHRAST_ERR_CUDA;
    k_pair_sums<<<(int)N, 256, 0, st>>>(pa);
    k_mean<<<1, 1024, 0, st>>>(pa);
    return cudaGetLastError() == cudaSuccess ? MESHRAST_OK : MESHRAST_ERR_CUDA;
}

MESHRAST_API int chamfer_bwd(const float *p, int64_t P1, const int64_t *first1, const int64_t *len1,
                             const float *q, int64_t P2, const int64_t *first2, const int64_t *len2, int64_t N,
                             int32_t D, const int64_t *idx_pq, const int64_t *idx_qp, const float *grad_loss,
                             const float *grad_per_pair, float *grad_p, float *grad_q, void *stream) {
    if (N < 0 || N > INT_MAX - 1 || P1 < 0 || P2 < 0 || D < 1 || D > 4) return MESHRAST_ERR_INVALID_ARG;
    if (N > 0 && (!first1 || !len1 || !first2 || !len2)) return MESHRAST_ERR_INVALID_ARG;
    if ((P1 > 0 && (!p || !idx_pq || !grad_p)) || (P2 > 0 && (!q || !idx_qp || !grad_q)))
        return MESHRAST_ERR_INVALID_ARG;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (P1 > 0 && cudaMemsetAsync(grad_p, 0, (size_t)P1 * D * sizeof(float), st) != cudaSuccess)
        return MESHRAST_ERR_CUDA;
    if (P2 > 0 && cudaMemsetAsync(grad_q, 0, (size_t)P2 * D * sizeof(float), st) != cudaSuccess)
        return MESHRAST_ERR_CUDA;
    if (N == 0 || P1 + P2 == 0) return MESHRAST_OK;
    ChamferBwdArgs a{p, q, first1, len1, first2, len2, idx_pq, idx_qp, grad_loss, grad_per_pair, grad_p, grad_q,
                     P1, P2, (int)N};
    const long long blocks = (P1 + P2 + 255) / 256;
    if (blocks > INT_MAX) return MESHRAST_ERR_INVALID_ARG;
    switch (D) {
        case 1: k_chamfer_bwd<1><<<(int)blocks, 256, 0, st>>>(a); break;
        case 2: k_chamfer_bwd<2><<<(int)blocks, 256, 0, st>>>(a); break;
        case 3: k_chamfer_bwd<3><<<(int)blocks, 256, 0, st>>>(a); break;
        default: k_chamfer_bwd<4><<<(int)blocks, 256, 0, st>>>(a); break;
    }
    return cudaGetLastError() == cudaSuccess ? MESHRAST_OK : MESHRAST_ERR_CUDA;
}

}  // extern "C"
