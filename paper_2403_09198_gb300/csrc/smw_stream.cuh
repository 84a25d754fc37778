// smw_stream.cuh -- row groups of the structured block-Jacobi apply streams
// (kernels_smw.cu).  A stream is a sequence of sections (runs of rows of one
// width); rows are packed in groups of whole 16-byte vectors of VEC = 16 /
// sizeof(T) positions, a group never straddles a chunk, and a lane reads VEC
// consecutive positions with one 16-byte shared-memory load.
#pragma once

#include "ring.cuh"
#include "sts_internal.h"

namespace sts {

__host__ __device__ constexpr int sap_gcd(int a, int b) { return b == 0 ? a : sap_gcd(b, a % b); }
// rows per group for rows of `width` positions, VEC positions per vector
__host__ __device__ constexpr int sap_rows(int width, int vec) { return vec / sap_gcd(width, vec); }
__host__ __device__ constexpr int sap_round(int n, int vec) { return (n + vec - 1) / vec * vec; }

// One group of G positions in registers (G / VEC 16-byte loads).
template <typename T, int G>
struct Group {
    using V = typename Vec16<T>::type;
    static constexpr int VEC = 16 / (int)sizeof(T), NV = G / VEC;
    static_assert(G % VEC == 0, "a group is whole vectors");
    V v[NV];
    __device__ __forceinline__ void load(const T *p) {
        const V *q = reinterpret_cast<const V *>(p);
#pragma unroll
        for (int j = 0; j < NV; ++j) v[j] = q[j * kTile];
    }
    __device__ __forceinline__ T operator[](int k) const { return vel(v[k / VEC], k % VEC); }
};

// One section of rows (forward level rows, backward level rows or tail) in
// groups of U rows of G stream positions.  The next group's coefficients and
// working-vector entries are loaded into registers before the current group
// is processed.  wsval(j): the working-vector value read for section row j
// (shared or global memory); row(g, w, u, j): computes section row j (row u of
// group g, working-vector value w) and returns its result; put(j, v) stores
// the result of section row j, one row late, when its FP64 FMA has long
// completed.
template <typename T, int G, int U, typename RingT, typename WsVal, typename RowF, typename PutF>
__device__ __forceinline__ void sap_section(RingT &R, int nrows, WsVal wsval, RowF row, PutF put) {
    const int ng = (nrows + U - 1) / U, nfull = nrows / U;
    Group<T, G> gA, gB;
    T xa[U], xb[U];
    T carry = T(0);
    auto load = [&](Group<T, G> &g, T (&xv)[U], int grp) {
        g.load(R.take(G));
#pragma unroll
        for (int u = 0; u < U; ++u) xv[u] = wsval(grp * U + u);
    };
    auto proc = [&](const Group<T, G> &g, const T (&xv)[U], int grp) {
        T prev = carry;
        if (grp < nfull) {
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const T v = row(g, xv[u], u, grp * U + u);
                if (u > 0 || grp > 0) put(grp * U + u - 1, prev);
                prev = v;
            }
        } else {
#pragma unroll
            for (int u = 0; u < U; ++u)
                if (grp * U + u < nrows) {
                    const T v = row(g, xv[u], u, grp * U + u);
                    if (u > 0 || grp > 0) put(grp * U + u - 1, prev);
                    prev = v;
                }
        }
        carry = prev;
    };
    if (nrows <= 0) return;
    load(gA, xa, 0);
    for (int grp = 0; grp < ng; grp += 2) {
        if (grp + 1 < ng) load(gB, xb, grp + 1);
        proc(gA, xa, grp);
        if (grp + 1 >= ng) break;
        if (grp + 2 < ng) load(gA, xa, grp + 2);
        proc(gB, xb, grp + 1);
    }
    put(nrows - 1, carry);
}


}  // namespace sts
