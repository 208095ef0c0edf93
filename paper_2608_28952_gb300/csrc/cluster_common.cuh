// cluster_common.cuh -- a packed symmetric matrix distributed over the
// shared memory of a thread-block cluster (used by the pivot-solve cluster
// kernel and the batched cluster kernel).
#pragma once
#include <cuda_runtime.h>

#include "jacobi_core.cuh"

namespace jac {

constexpr int PC_MAXC = 16;

// Row ranges: CTA r owns rows [row0[r], row0[r+1]) of the packed triangle,
// chosen so the entry counts are as equal as possible.
struct Split {
    int C;
    int row0[PC_MAXC + 1];
    int base[PC_MAXC + 1];  // packed index of the first entry of row0[r]
};

__host__ __device__ inline void make_split(int k, int C, Split& s)
{
    s.C = C;
    const long long total = (long long)k * (k + 1) / 2;
    int row = 0;
    s.row0[0] = 0;
    s.base[0] = 0;
    for (int r = 1; r < C; ++r) {
        const long long target = total * r / C;
        while (row < k && (long long)(row + 1) * (row + 2) / 2 <= target) ++row;
        s.row0[r] = row;
        s.base[r] = row * (row + 1) / 2;
    }
    s.row0[C] = k;
    s.base[C] = (int)total;
}

__host__ inline int split_max_chunk(int k, int C)
{
    Split s;
    make_split(k, C, s);
    int m = 0;
    for (int r = 0; r < C; ++r) m = s.base[r + 1] - s.base[r] > m ? s.base[r + 1] - s.base[r] : m;
    return m;
}

// Entry (i, j) of the distributed packed lower triangle; MAXC bounds the
// owner search (the cluster size C <= MAXC).
template <typename T, int MAXC>
struct DistPacked {
    T* ptr[MAXC];      // each CTA's chunk, as generic (DSMEM) addresses
    Split sp;
    __device__ __forceinline__ T* at(int i, int j) const
    {
        if (i < j) { const int t = i; i = j; j = t; }
        int r = 0;
#pragma unroll
        for (int u = 1; u < MAXC; ++u)
            if (u < sp.C && i >= sp.row0[u]) r = u;
        return ptr[r] + (tri(i) + j - sp.base[r]);
    }
};

// The same distribution addressed arithmetically: rinfo[i] (in the local
// shared memory of every CTA) = owner rank of row i << 20 | local element
// offset of entry (i, 0); the chunk sits at the same shared-memory offset in
// every CTA, so entry (i, j), j <= i, is `mapa` of the local address to the
// owner's window.  Loads and stores go through ld/st.shared::cluster.
template <typename T>
struct DistRows {
    uint32_t base;       // shared::cta address of the chunk
    const int* rinfo;
    __device__ __forceinline__ uint32_t addr(int i, int j) const
    {
        if (i < j) { const int t = i; i = j; j = t; }
        const int ri = rinfo[i];
        const uint32_t local = base + (uint32_t)(((ri & 0xFFFFF) + j) * (int)sizeof(T));
        uint32_t out;
        asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(out) : "r"(local), "r"(ri >> 20));
        return out;
    }
};

__device__ __forceinline__ float dsm_ld(uint32_t a, float)
{
    float v;
    asm volatile("ld.shared::cluster.f32 %0, [%1];" : "=f"(v) : "r"(a));
    return v;
}
__device__ __forceinline__ double dsm_ld(uint32_t a, double)
{
    double v;
    asm volatile("ld.shared::cluster.f64 %0, [%1];" : "=d"(v) : "r"(a));
    return v;
}
__device__ __forceinline__ void dsm_st(uint32_t a, float v)
{
    asm volatile("st.shared::cluster.f32 [%0], %1;" ::"r"(a), "f"(v));
}
__device__ __forceinline__ void dsm_st(uint32_t a, double v)
{
    asm volatile("st.shared::cluster.f64 [%0], %1;" ::"r"(a), "d"(v));
}

// Quad index qi -> (e1 < e2) in the order of build_quad_table (by e2, then e1).
__device__ __forceinline__ void quad_decode(int qi, int& e1, int& e2)
{
    int t = (int)((1.0f + sqrtf(1.0f + 8.0f * (float)qi)) * 0.5f);
    while (t * (t - 1) / 2 > qi) --t;
    while ((t + 1) * t / 2 <= qi) ++t;
    e2 = t;
    e1 = qi - t * (t - 1) / 2;
}

}  // namespace jac
