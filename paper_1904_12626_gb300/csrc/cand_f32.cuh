// cand_f32.cuh -- keys of the FP32-mixed path: candidates with certified bounds.
//
// The FP32 recurrence gives, for every cell, an upper bound U of the exact
// correlation (its covariance carries a bias equal to an error bound) and a
// lower bound L = U - 2 * bias * invn_i * invn_j.  A key holds one candidate
// neighbour per index together with such a pair:
//   hi = ord32(V) << 32 | (0xFFFFFFFF - idx)   V: upper bound, or the exact value
//   lo = ord32(L) << 32                          L: lower bound (L == V: exact)
// (hi == 0: no candidate yet; a real hi is never 0 because idx < 2^32 - 1).
// The two words are read with two plain loads, so a reader may see a torn
// pair (one word from before a concurrent update, one from after).  Every
// decision taken from a peeked key is either conservative for any mix of two
// successive key states (L never decreases) or is committed by a 128-bit CAS
// whose expected value is the peeked pair, which fails on a torn pair.  An
// index is only ever taken from hi, which is read whole.  A new candidate c is
//   discarded   if c.V <  key.L   (it cannot beat the key's candidate),
//   taken over  if c.L >  key.V   (it surely beats it),
//   compared exactly otherwise (its and/or the key's exact correlation is
//   computed in FP64 and the larger one, lower index on ties, is kept).
// L never decreases and bounds from below the exact value of the kept
// candidate, so every discarded candidate is no better than the final one:
// the final candidate is the exact argmax although most candidates are never
// computed exactly.  Only near-ties cost an exact dot product.
#pragma once

#include "internal.cuh"

namespace mpgb {

struct Cand {
    float V, L;
    long long idx;
};

enum { kDiscard = 0, kReplace = 1, kNeedCand = 2, kNeedKey = 4 };

__device__ __forceinline__ unsigned f2o(float f) { return ord32(__float_as_uint(f + 0.0f)); }
__device__ __forceinline__ float o2f(unsigned o) { return __uint_as_float(unord32(o)); }

__device__ __forceinline__ Key128 cand_key(const Cand &c)
{
    Key128 k;
    k.hi = ((unsigned long long)f2o(c.V) << 32) | (unsigned long long)(0xFFFFFFFFu - (unsigned)c.idx);
    k.lo = (unsigned long long)f2o(c.L) << 32;
    return k;
}
__device__ __forceinline__ bool key_empty(const Key128 &k) { return k.hi == 0ull; }
__device__ __forceinline__ bool key_same(const Key128 &a, const Key128 &b)
{
    return a.hi == b.hi && a.lo == b.lo;
}
__device__ __forceinline__ Cand key_cand(const Key128 &k)
{
    Cand c;
    c.V = o2f((unsigned)(k.hi >> 32));
    c.L = o2f((unsigned)(k.lo >> 32));
    c.idx = (long long)(0xFFFFFFFFu - (unsigned)(k.hi & 0xFFFFFFFFull));
    return c;
}
__device__ __forceinline__ Key128 key_peek(const Key128 *p)
{
    Key128 k;
    k.hi = __ldcg(&p->hi);
    k.lo = __ldcg(&p->lo);
    return k;
}

// Decision for candidate c against key k.  kx is the exact correlation of the
// key's candidate when already computed for index kx_idx (else kx_idx < 0).
__device__ __forceinline__ int classify(const Cand &c, const Key128 &k, float kx, long long kx_idx)
{
    if (key_empty(k)) return kReplace;
    Cand q = key_cand(k);
    if (q.L != q.V && q.idx == kx_idx) q.V = q.L = kx;
    if (c.V < q.L) return kDiscard;
    if (c.L > q.V) return kReplace;
    const bool ce = c.L == c.V, qe = q.L == q.V;
    if (ce && qe) {
        const unsigned long long a = ((unsigned long long)f2o(c.V) << 32) |
                                     (0xFFFFFFFFu - (unsigned)c.idx);
        const unsigned long long b = ((unsigned long long)f2o(q.V) << 32) |
                                     (0xFFFFFFFFu - (unsigned)q.idx);
        return a > b ? kReplace : kDiscard;
    }
    return (ce ? 0 : kNeedCand) | (qe ? 0 : kNeedKey);
}

__device__ __forceinline__ void raise_thr(float4 *g, float4 *sm, float L)
{
    if (sm && L > sm->w) sm->w = L;
    if (L > g->w) g->w = L;
}

}  // namespace mpgb
