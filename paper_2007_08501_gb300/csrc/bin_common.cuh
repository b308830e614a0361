// Device helpers shared by the mesh and point rasterizers: camera projection
// in double-float, binning rectangles, the front-to-back sort of a bin's
// entries and the shared-memory K-nearest lists.
#pragma once

#include "rast_common.cuh"

namespace mr {

__device__ __forceinline__ int find_mesh(const int64_t *first_face, int N, int64_t f) {
    int lo = 0, hi = N - 1, ans = -1;
    while (lo <= hi) {
        int mid = (lo + hi) >> 1;
        if (first_face[mid] <= f) { ans = mid; lo = mid + 1; } else { hi = mid - 1; }
    }
    return ans;
}

// Image of element i of a packed batch (ranges first[n] .. first[n] + num[n]),
// or -1.  Thread 0 looks up the block's first element once; threads whose
// element lies in that image's range skip their own binary search.  Every
// thread of the block must call it (it synchronises the block).
__device__ __forceinline__ int block_find_mesh(const int64_t *first, const int64_t *num, int N, int64_t count,
                                               int64_t i) {
    __shared__ int s_n;
    __shared__ long long s_lo, s_hi;
    if (threadIdx.x == 0) {
        const int64_t i0 = (int64_t)blockIdx.x * blockDim.x;
        const int n0 = i0 < count ? find_mesh(first, N, i0) : -1;
        s_n = n0;
        s_lo = n0 >= 0 ? first[n0] : 0;
        s_hi = n0 >= 0 ? first[n0] + num[n0] : 0;
    }
    __syncthreads();
    if (i >= count) return -1;
    if (s_n >= 0 && i >= s_lo && i < s_hi) return s_n;
    const int n = find_mesh(first, N, i);
    return (n >= 0 && i < first[n] + num[n]) ? n : -1;
}

// world -> view -> NDC of one corner, in double-float arithmetic
__device__ __forceinline__ void project_corner(const float *cam, float px, float py, float pz, df &X, df &Y,
                                               df &Z) {
    df d0 = two_sum(px, -cam[9]), d1 = two_sum(py, -cam[10]), d2 = two_sum(pz, -cam[11]);
    df x = df_add(df_add(df_mul_f(d0, cam[0]), df_mul_f(d1, cam[1])), df_mul_f(d2, cam[2]));
    df y = df_add(df_add(df_mul_f(d0, cam[3]), df_mul_f(d1, cam[4])), df_mul_f(d2, cam[5]));
    df z = df_add(df_add(df_mul_f(d0, cam[6]), df_mul_f(d1, cam[7])), df_mul_f(d2, cam[8]));
    float f = cam[12];
    X = df_div(df_mul_f(x, f), z);
    Y = df_div(df_mul_f(y, f), z);
    Z = z;
}

__device__ __forceinline__ df df_min(df a, df b) { return (a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo)) ? a : b; }
__device__ __forceinline__ df df_max(df a, df b) { return (a.hi > b.hi || (a.hi == b.hi && a.lo > b.lo)) ? a : b; }

// Columns (or rows) whose fp32 pixel centre lies in [lo, hi]: first index
// with centre <= hi, last index with centre >= lo (centres decrease with the
// index).  Exactly the comparisons the fine pass makes.
__device__ __forceinline__ float pc_hi(int i, int S) {
    float h, l;
    pix_coord(i, S, h, l);
    return h;
}
__device__ __forceinline__ void centre_range(float lo, float hi, int S, int &i0, int &i1) {
    float Sf = (float)S;
    int a = (int)ceilf(fminf(fmaxf(((Sf - 1.f) - hi * Sf) * 0.5f, -1.f), Sf));
    a = max(0, min(a, S));
    while (a > 0 && pc_hi(a - 1, S) <= hi) --a;
    while (a < S && pc_hi(a, S) > hi) ++a;
    int b = (int)floorf(fminf(fmaxf(((Sf - 1.f) - lo * Sf) * 0.5f, -1.f), Sf));
    b = max(-1, min(b, S - 1));
    while (b < S - 1 && pc_hi(b + 1, S) >= lo) ++b;
    while (b >= 0 && pc_hi(b, S) < lo) --b;
    i0 = a;
    i1 = b;
}

// Bins (bx0..bx1, by0..by1) whose pixel-centre span meets the box (xmin,
// xmax, ymin, ymax).  Empty when bx0 > bx1 or by0 > by1.
__device__ __forceinline__ void bin_rect_box(const float4 &box, int S, int bin, int &bx0, int &bx1, int &by0,
                                             int &by1) {
    if (!(box.x <= box.y) || !(box.z <= box.w)) { bx0 = 1; bx1 = 0; by0 = 1; by1 = 0; return; }
    int c0, c1, r0, r1;
    centre_range(box.x, box.y, S, c0, c1);
    centre_range(box.z, box.w, S, r0, r1);
    if (c0 > S - 1 || c1 < 0 || r0 > S - 1 || r1 < 0) { bx0 = 1; bx1 = 0; by0 = 1; by1 = 0; return; }
    bx0 = c0 / bin;
    bx1 = c1 / bin;
    by0 = r0 / bin;
    by1 = r1 / bin;
}

// Bins of a face: the bin's pixel-centre span meets the inflated bbox.
__device__ __forceinline__ void bin_rect(const FaceRec &R, int S, int bin, int &bx0, int &bx1, int &by0,
                                         int &by1) {
    bin_rect_box(R.c, S, bin, bx0, bx1, by0, by1);
}

// Bitonic sort of N2 = BD * E entries, E consecutive entries per thread in
// registers: stages whose partner is in the same thread (distance < E) run in
// registers, stages whose partner is in the same warp (distance < 32 E) go
// through lane shuffles, and only the few wider ones through shared memory
// (two barriers each).  Padding entries (all ones) sort last.
template <int E, int J>
__device__ __forceinline__ void sort_stage_local(unsigned long long (&v)[E], int k2, int tid) {
#pragma unroll
    for (int e = 0; e < E; ++e) {
        if (e & J) continue;
        const int i = tid * E + e;
        const unsigned long long x = v[e], y = v[e + J];
        const bool asc = (i & k2) == 0;
        const unsigned long long lo = x < y ? x : y, hi = x < y ? y : x;
        v[e] = asc ? lo : hi;
        v[e + J] = asc ? hi : lo;
    }
}

template <int BD, int E>
__device__ __forceinline__ void sort_entries_regs(unsigned long long *s_sort, const unsigned long long *src, int m) {
    constexpr int N2 = BD * E;
    const int tid = threadIdx.x;
    unsigned long long v[E];
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const int i = tid * E + e;
        v[e] = i < m ? src[i] : ~0ull;
    }
#pragma unroll 1
    for (int k2 = 2; k2 <= N2; k2 <<= 1) {
#pragma unroll 1
        for (int j2 = k2 >> 1; j2 > 0; j2 >>= 1) {
            if (j2 < E) {
                if constexpr (E > 4) { if (j2 == 4) { sort_stage_local<E, (E > 4 ? 4 : 1)>(v, k2, tid); continue; } }
                if constexpr (E > 2) { if (j2 == 2) { sort_stage_local<E, (E > 2 ? 2 : 1)>(v, k2, tid); continue; } }
                sort_stage_local<E, 1>(v, k2, tid);
                continue;
            }
            if (j2 < 32 * E) {
                const int lm = j2 / E;  // partner lane distance
#pragma unroll
                for (int e = 0; e < E; ++e) {
                    const int i = tid * E + e;
                    const unsigned long long o = __shfl_xor_sync(0xffffffffu, v[e], lm);
                    const bool keep_min = ((i & j2) == 0) == ((i & k2) == 0);
                    v[e] = keep_min ? (o < v[e] ? o : v[e]) : (o > v[e] ? o : v[e]);
                }
                continue;
            }
#pragma unroll
            for (int e = 0; e < E; ++e) s_sort[tid * E + e] = v[e];
            __syncthreads();
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const int i = tid * E + e;
                const unsigned long long o = s_sort[i ^ j2];
                const bool keep_min = ((i & j2) == 0) == ((i & k2) == 0);
                v[e] = keep_min ? (o < v[e] ? o : v[e]) : (o > v[e] ? o : v[e]);
            }
            __syncthreads();
        }
    }
#pragma unroll
    for (int e = 0; e < E; ++e) s_sort[tid * E + e] = v[e];
    __syncthreads();
}

// Sorts m <= sort-buffer bin entries (64-bit keys) from src into s_sort,
// ascending; every thread of the block (BD threads) must call it.  A segment
// that fits one entry per thread sorts in registers: partners closer than 32
// trade through shuffles, farther ones through shared memory.  Larger ones
// run a bitonic sort in shared memory.  Padding entries (all ones) sort last.
template <int BD, bool REGS = false>
__device__ __forceinline__ void sort_entries(unsigned long long *s_sort, const unsigned long long *src, int m) {
    const int tid = threadIdx.x;
    int n2 = 32;
    while (n2 < m) n2 <<= 1;
    if (n2 <= BD) {
        // one entry per thread: partners closer than 32 trade through
        // shuffles, farther ones through shared memory
        unsigned long long v = tid < m ? src[tid] : ~0ull;
#pragma unroll 1
        for (int k2 = 2; k2 <= n2; k2 <<= 1) {
#pragma unroll 1
            for (int j2 = k2 >> 1; j2 > 0; j2 >>= 1) {
                unsigned long long o;
                if (j2 >= 32) {
                    s_sort[tid] = v;
                    __syncthreads();
                    o = s_sort[tid ^ j2];
                    __syncthreads();
                } else {
                    o = __shfl_xor_sync(0xffffffffu, v, j2);
                }
                const bool keep_min = ((tid & j2) == 0) == ((tid & k2) == 0);
                v = keep_min ? (o < v ? o : v) : (o > v ? o : v);
            }
        }
        s_sort[tid] = v;
        __syncthreads();
        return;
    }
    // REGS: two to eight entries per thread in registers and shuffles (more
    // registers, far fewer barriers)
    if constexpr (REGS) {
        if (n2 == 2 * BD) { sort_entries_regs<BD, 2>(s_sort, src, m); return; }
        if (n2 == 4 * BD) { sort_entries_regs<BD, 4>(s_sort, src, m); return; }
        if (n2 == 8 * BD) { sort_entries_regs<BD, 8>(s_sort, src, m); return; }
    }
    for (int i = tid; i < n2; i += BD) s_sort[i] = i < m ? src[i] : ~0ull;
    __syncthreads();
    // bitonic sort in shared memory (padding entries sort last)
#pragma unroll 1
    for (int k2 = 2; k2 <= n2; k2 <<= 1) {
#pragma unroll 1
        for (int j2 = k2 >> 1; j2 > 0; j2 >>= 1) {
            for (int i = tid; i < (n2 >> 1); i += BD) {
                const int lo = ((i & ~(j2 - 1)) << 1) | (i & (j2 - 1));
                const int hi = lo + j2;
                const unsigned long long x = s_sort[lo], y = s_sort[hi];
                if ((x > y) == ((lo & k2) == 0)) {
                    s_sort[lo] = y;
                    s_sort[hi] = x;
                }
            }
            __syncthreads();
        }
    }
}

// large-K variant: per-thread sorted lists in shared memory; element k of a
// thread's list sits at z[k * stride], f[k * stride]
struct SmemTopK {
    float *z;
    int *f;
    int stride, K;
    int n;  // entries held (< K while the list is not full)
    __device__ __forceinline__ void init() { n = 0; }
    // K-th smallest depth so far (infinite until K candidates were kept)
    __device__ __forceinline__ float thr() const {
        return n < K ? __int_as_float(0x7f800000) : z[(K - 1) * stride];
    }
    __device__ __forceinline__ bool admits(float zz, int ff) const {
        return n < K || key_less(zz, ff, z[(K - 1) * stride], f[(K - 1) * stride]);
    }
    // insertion from the end of the held entries: candidates arrive nearly in
    // depth order, so most insertions are appends
    __device__ __forceinline__ void insert(float zz, int ff) {
        int k = n < K ? n : K - 1;
        while (k > 0) {
            float zp = z[(k - 1) * stride];
            int fp = f[(k - 1) * stride];
            if (!key_less(zz, ff, zp, fp)) break;
            z[k * stride] = zp;
            f[k * stride] = fp;
            --k;
        }
        z[k * stride] = zz;
        f[k * stride] = ff;
        if (n < K) ++n;
    }
};

}  // namespace mr
