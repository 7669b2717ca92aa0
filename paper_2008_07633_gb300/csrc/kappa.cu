// Relative condition number kappa(L_G, L_P) of Sec. 2.2 (Eq. eqn:ineq): the ratio of the largest
// to the smallest generalised eigenvalue of L_G x = lambda L_P x on the complement of the common
// null space (P spans the components of G, so both null spaces are the per-component constants).
// It is the paper's measure of sparsifier quality, used here to check the method; it is not on the
// filter+score path.
//
// Method (not in the paper, which only reports kappa):
//  * Lanczos on A = L_P^+ L_G, self-adjoint in the L_P inner product, in FP64 with full
//    reorthogonalisation (classical Gram-Schmidt applied twice). Vectors v_j and u_j = L_P v_j are
//    kept; u_{j+1} is recomputed by one product with L_P each step (carried by the recurrence it
//    drifts out of the range of L_P). Every vector is grounded (its value at one representative
//    node per component subtracted), since null-space components, invisible to the L_P norm,
//    would otherwise be amplified by 1 / beta at every step.
//  * Each L_P solve is exact up to FP64 rounding: a factorisation eliminates nodes of degree <= 2
//    in rounds (a leaf folds into its neighbour; a degree-2 node becomes the series edge
//    w_a w_b / (w_a + w_b) between its neighbours). Each round eliminates an independent set of
//    such nodes chosen by a seeded priority, so a tree or a chain takes O(log n) rounds. What is
//    left (the core: min degree 3, at most about 2x the edges beyond a spanning forest) is solved
//    by Jacobi-preconditioned CG to a relative residual of 1e-13 (or 1e-12 of the whole
//    right-hand side). The right-hand side is folded
//    forward round by round and the solution substituted back in reverse.
//  * The extreme eigenvalues of the Lanczos tridiagonal matrix come from bisection on Sturm
//    counts (one thread, FP64). lambda_min is exactly 1 when G \ P has more components than G
//    (then no Lanczos estimate is needed for it), which holds for sparsifiers that leave some
//    node untouched by the dropped edges.
// Every reduction has a fixed order (per-block partials folded in block order), so the result is
// deterministic.
#include <cmath>
#include <vector>

#include "sfg_internal.cuh"

namespace {

constexpr int kBlock = 256;
constexpr int kRedBlocks = 1024;  // partial sums per reduction (fixed: the fold order is fixed)
constexpr int kMaxRounds = 512;

template <typename K>
int grid_of(sfg_ctx* ctx, K kernel, int64_t work) {
    return sfg_grid(ctx, (const void*)kernel, kBlock, 0, work);
}

__device__ __forceinline__ double block_sum(double v, double* sh) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < kBlock / 32; ++w) s += sh[w];
    __syncthreads();
    return s;  // valid in thread 0
}

// FP32 -> FP64 copy (weights of the working edge list).
__global__ void k_widen(int64_t m, const float* __restrict__ a, double* __restrict__ b) {
    for (int64_t i = blockIdx.x * (int64_t)kBlock + threadIdx.x; i < m; i += (int64_t)gridDim.x * kBlock)
        b[i] = (double)a[i];
}

// Number of keys that are not ~0 (they sort last).
__global__ void k_count_valid(int64_t len, const uint64_t* __restrict__ key, int64_t* __restrict__ out) {
    if (threadIdx.x != 0) return;
    int64_t lo = 0, hi = len;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (key[mid] != ~0ull) lo = mid + 1; else hi = mid;
    }
    *out = lo;
}

// ---------------------------------------------------------------- factorisation of L_P ----------

// Alive edges of node v, merged by neighbour: at most two distinct neighbours make v a candidate.
__global__ void k_el_scan(int32_t n, const int32_t* __restrict__ row_ptr,
                          const int32_t* __restrict__ adj, const int32_t* __restrict__ eu,
                          const int32_t* __restrict__ ev, const double* __restrict__ ew,
                          const uint8_t* __restrict__ ealive, const uint8_t* __restrict__ nalive,
                          uint8_t* __restrict__ cand, int32_t* __restrict__ nb0,
                          int32_t* __restrict__ nb1, double* __restrict__ w0,
                          double* __restrict__ w1) {
    for (int64_t v = blockIdx.x * (int64_t)kBlock + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * kBlock) {
        if (!nalive[v]) {
            cand[v] = 0;
            continue;
        }
        int32_t a = -1, b = -1;
        double wa = 0.0, wb = 0.0;
        bool more = false;
        for (int32_t s = row_ptr[v]; s < row_ptr[v + 1]; ++s) {
            const int32_t e = adj[s];
            if (!ealive[e]) continue;
            const int32_t o = eu[e] == (int32_t)v ? ev[e] : eu[e];
            if (o == a) wa += ew[e];
            else if (o == b) wb += ew[e];
            else if (a < 0) { a = o; wa = ew[e]; }
            else if (b < 0) { b = o; wb = ew[e]; }
            else { more = true; break; }
        }
        cand[v] = more ? 0 : 1;
        nb0[v] = a;
        nb1[v] = b;
        w0[v] = wa;
        w1[v] = wb;
    }
}

__device__ __forceinline__ uint64_t el_priority(int32_t v, int round) {
    return sfg_splitmix64(((uint64_t)round << 32) ^ (uint32_t)v);
}

// A candidate is eliminated when it outranks every candidate neighbour (priority, then id).
__global__ void k_el_choose(int32_t n, int round, const uint8_t* __restrict__ cand,
                            const int32_t* __restrict__ nb0, const int32_t* __restrict__ nb1,
                            uint8_t* __restrict__ chosen) {
    for (int64_t v = blockIdx.x * (int64_t)kBlock + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * kBlock) {
        uint8_t c = cand[v];
        if (c) {
            const uint64_t pv = el_priority((int32_t)v, round);
            const int32_t nbs[2] = {nb0[v], nb1[v]};
            for (int i = 0; i < 2; ++i) {
                const int32_t o = nbs[i];
                if (o < 0 || !cand[o]) continue;
                const uint64_t po = el_priority(o, round);
                if (po > pv || (po == pv && o > (int32_t)v)) c = 0;
            }
        }
        chosen[v] = c;
    }
}

// Eliminate the chosen nodes. A degree-2 node keeps its first edge to neighbour a, rewritten as
// the series edge (a, b), and hands it to b in place of its first edge to b; its other edges die.
// Chosen nodes are pairwise non-adjacent, so no two of them touch the same edge or slot.
// Contributions to the right-hand side fold are written as (round | target, entry) keys, entry =
// 2 * (position of v among this round's eliminations) + side, with coefficient w_side / (w_a + w_b).
__global__ void k_el_apply(int32_t n, int round, const uint8_t* __restrict__ chosen,
                           const int64_t* __restrict__ pos, int64_t base,
                           const int32_t* __restrict__ row_ptr, int32_t* __restrict__ adj,
                           int32_t* __restrict__ eu, int32_t* __restrict__ ev,
                           double* __restrict__ ew, uint8_t* __restrict__ ealive,
                           uint8_t* __restrict__ nalive, const int32_t* __restrict__ nb0,
                           const int32_t* __restrict__ nb1, const double* __restrict__ w0,
                           const double* __restrict__ w1, int32_t* __restrict__ order,
                           uint64_t* __restrict__ ckey, uint32_t* __restrict__ cval,
                           int32_t* __restrict__ csrc, double* __restrict__ ccoef) {
    for (int64_t v = blockIdx.x * (int64_t)kBlock + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * kBlock) {
        if (!chosen[v]) continue;
        const int64_t k = base + pos[v];  // global elimination index
        order[k] = (int32_t)v;
        nalive[v] = 0;
        const int32_t a = nb0[v], b = nb1[v];
        int32_t ea = -1, eb = -1;
        for (int32_t s = row_ptr[v]; s < row_ptr[v + 1]; ++s) {
            const int32_t e = adj[s];
            if (!ealive[e]) continue;
            const int32_t o = eu[e] == (int32_t)v ? ev[e] : eu[e];
            if (b >= 0 && o == a && ea < 0) { ea = e; continue; }  // kept as the series edge
            if (b >= 0 && o == b && eb < 0) eb = e;
            ealive[e] = 0;
        }
        const double wa = w0[v], wb = w1[v];
        for (int side = 0; side < 2; ++side) {
            const int32_t t = side ? b : a;
            const int64_t j = 2 * k + side;
            ckey[j] = t >= 0 ? ((uint64_t)round << 32) | (uint32_t)t : ~0ull;  // ~0: no entry
            cval[j] = (uint32_t)j;
            csrc[j] = (int32_t)v;
            ccoef[j] = b < 0 ? 1.0 : (side ? wb : wa) / (wa + wb);
        }
        if (b >= 0) {
            eu[ea] = a;
            ev[ea] = b;
            ew[ea] = wa * wb / (wa + wb);
            for (int32_t s = row_ptr[b]; s < row_ptr[b + 1]; ++s)
                if (adj[s] == eb) {
                    adj[s] = ea;
                    break;
                }
        }
    }
}

// Segment heads of the sorted contribution keys (one segment per (round, target)).
__global__ void k_el_heads(int64_t len, const uint64_t* __restrict__ key, uint8_t* __restrict__ head) {
    for (int64_t i = blockIdx.x * (int64_t)kBlock + threadIdx.x; i < len;
         i += (int64_t)gridDim.x * kBlock)
        head[i] = key[i] != ~0ull && (i == 0 || key[i] != key[i - 1]);
}

__global__ void k_el_segs(int64_t len, const uint64_t* __restrict__ key,
                          const uint8_t* __restrict__ head, const int64_t* __restrict__ hpos,
                          int64_t* __restrict__ seg_start, int32_t* __restrict__ seg_round,
                          int32_t* __restrict__ seg_target) {
    for (int64_t i = blockIdx.x * (int64_t)kBlock + threadIdx.x; i < len;
         i += (int64_t)gridDim.x * kBlock)
        if (head[i]) {
            seg_start[hpos[i]] = i;
            seg_round[hpos[i]] = (int32_t)(key[i] >> 32);
            seg_target[hpos[i]] = (int32_t)(key[i] & 0xffffffffu);
        }
}

// Core numbering and the core's directed entries (row, col) -> sorted into CSR by the caller.
__global__ void k_core_flag(int32_t n, const uint8_t* __restrict__ nalive, uint8_t* __restrict__ f) {
    for (int64_t v = blockIdx.x * (int64_t)kBlock + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * kBlock)
        f[v] = nalive[v];
}

__global__ void k_core_entries(int64_t m, const int32_t* __restrict__ eu,
                               const int32_t* __restrict__ ev, const uint8_t* __restrict__ ealive,
                               const int64_t* __restrict__ cid, const int64_t* __restrict__ epos,
                               uint64_t* __restrict__ key, uint32_t* __restrict__ val) {
    for (int64_t e = blockIdx.x * (int64_t)kBlock + threadIdx.x; e < m;
         e += (int64_t)gridDim.x * kBlock) {
        if (!ealive[e]) continue;
        const uint64_t a = (uint64_t)cid[eu[e]], b = (uint64_t)cid[ev[e]];
        const int64_t j = 2 * epos[e];
        key[j] = (a << 32) | b;
        val[j] = (uint32_t)e;
        key[j + 1] = (b << 32) | a;
        val[j + 1] = (uint32_t)e;
    }
}

__global__ void k_core_csr(int64_t len, int32_t nc, const uint64_t* __restrict__ key,
                           const uint32_t* __restrict__ val, const double* __restrict__ ew,
                           int64_t* __restrict__ rp, int32_t* __restrict__ col,
                           double* __restrict__ w) {
    for (int64_t i = blockIdx.x * (int64_t)kBlock + threadIdx.x; i < len;
         i += (int64_t)gridDim.x * kBlock) {
        const int32_t r = (int32_t)(key[i] >> 32);
        col[i] = (int32_t)(key[i] & 0xffffffffu);
        w[i] = ew[val[i]];
        const int32_t rprev = i == 0 ? -1 : (int32_t)(key[i - 1] >> 32);
        for (int32_t q = rprev + 1; q <= r; ++q) rp[q] = i;
        if (i == len - 1)
            for (int32_t q = r + 1; q <= nc; ++q) rp[q] = len;
    }
}

__global__ void k_core_diag(int32_t nc, const int64_t* __restrict__ rp, const double* __restrict__ w,
                            double* __restrict__ d) {
    for (int64_t i = blockIdx.x * (int64_t)kBlock + threadIdx.x; i < nc;
         i += (int64_t)gridDim.x * kBlock) {
        double s = 0.0;
        for (int64_t j = rp[i]; j < rp[i + 1]; ++j) s += w[j];
        d[i] = s;
    }
}

// ---------------------------------------------------------------- solve kernels -----------------

// Forward fold of one round: b[target] += sum over its entries (sorted order) of coef * b[src].
__global__ void k_sv_forward(int64_t s0, int64_t s1, const int64_t* __restrict__ seg_start,
                             const int32_t* __restrict__ seg_target, const uint32_t* __restrict__ cval,
                             const int32_t* __restrict__ csrc, const double* __restrict__ ccoef,
                             double* __restrict__ b) {
    for (int64_t s = s0 + blockIdx.x * (int64_t)kBlock + threadIdx.x; s < s1;
         s += (int64_t)gridDim.x * kBlock) {
        double acc = 0.0;
        for (int64_t i = seg_start[s]; i < seg_start[s + 1]; ++i) {
            const uint32_t j = cval[i];
            acc += ccoef[j] * b[csrc[j]];
        }
        b[seg_target[s]] += acc;
    }
}

// Back substitution of one round (nodes order[k0, k1)).
__global__ void k_sv_backward(int64_t k0, int64_t k1, const int32_t* __restrict__ order,
                              const int32_t* __restrict__ nb0, const int32_t* __restrict__ nb1,
                              const double* __restrict__ w0, const double* __restrict__ w1,
                              const double* __restrict__ b, double* __restrict__ x) {
    for (int64_t k = k0 + blockIdx.x * (int64_t)kBlock + threadIdx.x; k < k1;
         k += (int64_t)gridDim.x * kBlock) {
        const int32_t v = order[k], a = nb0[v], c = nb1[v];
        double xv = 0.0;  // a fully eliminated component is grounded at its last node
        if (c >= 0) xv = (b[v] + w0[v] * x[a] + w1[v] * x[c]) / (w0[v] + w1[v]);
        else if (a >= 0) xv = x[a] + b[v] / w0[v];
        x[v] = xv;
    }
}

__global__ void k_gather(int32_t nc, const int32_t* __restrict__ core_nodes,
                         const double* __restrict__ b, double* __restrict__ bc) {
    for (int64_t i = blockIdx.x * (int64_t)kBlock + threadIdx.x; i < nc;
         i += (int64_t)gridDim.x * kBlock)
        bc[i] = b[core_nodes[i]];
}

__global__ void k_scatter(int32_t nc, const int32_t* __restrict__ core_nodes,
                          const double* __restrict__ xc, double* __restrict__ x) {
    for (int64_t i = blockIdx.x * (int64_t)kBlock + threadIdx.x; i < nc;
         i += (int64_t)gridDim.x * kBlock)
        x[core_nodes[i]] = xc[i];
}

__global__ void k_core_nodes(int32_t n, const uint8_t* __restrict__ nalive,
                             const int64_t* __restrict__ cid, int32_t* __restrict__ core_nodes) {
    for (int64_t v = blockIdx.x * (int64_t)kBlock + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * kBlock)
        if (nalive[v]) core_nodes[cid[v]] = (int32_t)v;
}

// Jacobi-preconditioned CG on the core. Scalars live on the device: sc[0] = rho, sc[1] = alpha,
// sc[2] = beta, sc[3] = r.r, sc[4] = b.b, sc[5] = |whole right-hand side|^2, sc[6] = the squared
// tolerance, sc[7] = done. The core Laplacian is singular: past convergence CG drifts along its
// null space and the residual grows again, so the fold that first sees r.r <= tolerance sets
// `done` and every later CG kernel returns at once, keeping that iterate.
__global__ void k_cg_init(int32_t nc, const double* __restrict__ b, const double* __restrict__ d,
                          double* __restrict__ x, double* __restrict__ r, double* __restrict__ p,
                          double* __restrict__ part) {
    __shared__ double sh[kBlock / 32];
    double s_rz = 0.0, s_bb = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)kBlock + threadIdx.x; i < nc;
         i += (int64_t)gridDim.x * kBlock) {
        const double bi = b[i], z = d[i] > 0.0 ? bi / d[i] : 0.0;
        x[i] = 0.0;
        r[i] = bi;
        p[i] = z;
        s_rz += bi * z;
        s_bb += bi * bi;
    }
    s_rz = block_sum(s_rz, sh);
    s_bb = block_sum(s_bb, sh);
    if (threadIdx.x == 0) {
        part[blockIdx.x] = s_rz;
        part[kRedBlocks + blockIdx.x] = s_bb;
    }
}

// Fold `nsum` partial arrays (each of gridDim of the producing kernel, padded to kRedBlocks) in
// block order; mode 0: rho = s0, bb = s1, rr = s1; mode 1: alpha = rho / s0; mode 2: beta =
// s0 / rho, rho = s0, rr = s1.
__global__ void k_cg_fold(const double* __restrict__ part, int nparts, int mode, double* __restrict__ sc) {
    __shared__ double sh[kBlock / 32];
    if (mode != 0 && sc[7] != 0.0) return;
    double s0 = 0.0, s1 = 0.0;
    for (int i = threadIdx.x; i < nparts; i += kBlock) {  // fixed assignment and order
        s0 += part[i];
        s1 += part[kRedBlocks + i];
    }
    s0 = block_sum(s0, sh);
    s1 = block_sum(s1, sh);
    if (threadIdx.x == 0) {
        if (mode == 0) {
            sc[0] = s0;
            sc[4] = s1;
            sc[3] = s1;
            // relative residual 1e-13 of the core's right-hand side, or 1e-12 of the whole one
            // (the core part can be tiny, and rounding in the forward fold leaves it slightly
            // inconsistent)
            sc[6] = fmax(1e-26 * s1, 1e-24 * sc[5]);
            sc[7] = s1 <= sc[6] ? 1.0 : 0.0;
        } else if (mode == 1) {
            sc[1] = s0 != 0.0 ? sc[0] / s0 : 0.0;
        } else {
            sc[2] = sc[0] != 0.0 ? s0 / sc[0] : 0.0;
            sc[0] = s0;
            sc[3] = s1;
            if (s1 <= sc[6] || !(s1 == s1)) sc[7] = 1.0;
        }
    }
}

__global__ void k_cg_spmv(int32_t nc, const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                          const double* __restrict__ w, const double* __restrict__ d,
                          const double* __restrict__ p, double* __restrict__ q,
                          double* __restrict__ part, const double* __restrict__ sc) {
    __shared__ double sh[kBlock / 32];
    if (sc[7] != 0.0) return;
    double s = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)kBlock + threadIdx.x; i < nc;
         i += (int64_t)gridDim.x * kBlock) {
        double a = 0.0;
        for (int64_t j = rp[i]; j < rp[i + 1]; ++j) a += w[j] * p[col[j]];
        const double qi = d[i] * p[i] - a;
        q[i] = qi;
        s += p[i] * qi;
    }
    s = block_sum(s, sh);
    if (threadIdx.x == 0) {
        part[blockIdx.x] = s;
        part[kRedBlocks + blockIdx.x] = 0.0;
    }
}

__global__ void k_cg_update(int32_t nc, const double* __restrict__ sc, const double* __restrict__ d,
                            const double* __restrict__ p, const double* __restrict__ q,
                            double* __restrict__ x, double* __restrict__ r, double* __restrict__ z,
                            double* __restrict__ part) {
    __shared__ double sh[kBlock / 32];
    if (sc[7] != 0.0) return;
    const double alpha = sc[1];
    double s_rz = 0.0, s_rr = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)kBlock + threadIdx.x; i < nc;
         i += (int64_t)gridDim.x * kBlock) {
        x[i] += alpha * p[i];
        const double ri = r[i] - alpha * q[i];
        r[i] = ri;
        const double zi = d[i] > 0.0 ? ri / d[i] : 0.0;
        z[i] = zi;
        s_rz += ri * zi;
        s_rr += ri * ri;
    }
    s_rz = block_sum(s_rz, sh);
    s_rr = block_sum(s_rr, sh);
    if (threadIdx.x == 0) {
        part[blockIdx.x] = s_rz;
        part[kRedBlocks + blockIdx.x] = s_rr;
    }
}

__global__ void k_cg_dir(int32_t nc, const double* __restrict__ sc, const double* __restrict__ z,
                         double* __restrict__ p) {
    if (sc[7] != 0.0) return;
    const double beta = sc[2];
    for (int64_t i = blockIdx.x * (int64_t)kBlock + threadIdx.x; i < nc;
         i += (int64_t)gridDim.x * kBlock)
        p[i] = z[i] + beta * p[i];
}

// ---------------------------------------------------------------- Lanczos kernels ---------------

// y = L x (FP64) for a CSR Laplacian with FP32 weights and FP64 degrees.
__global__ void k_lap_mul(int32_t n, const int32_t* __restrict__ row_ptr,
                          const int2* __restrict__ colval, const double* __restrict__ deg,
                          const double* __restrict__ x, double* __restrict__ y) {
    for (int64_t i = blockIdx.x * (int64_t)kBlock + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * kBlock) {
        double a = 0.0;
        for (int32_t j = row_ptr[i]; j < row_ptr[i + 1]; ++j)
            a += (double)__int_as_float(colval[j].y) * x[colval[j].x];
        y[i] = deg[i] * x[i] - a;
    }
}

// Partial dot products of w with vectors 0..nv-1 of the column block M (n x nv, vector i at
// M + i * n): part[i * kRedBlocks + block].
__global__ void k_multidot(int64_t n, int nv, const double* __restrict__ M,
                           const double* __restrict__ w, double* __restrict__ part) {
    __shared__ double sh[kBlock / 32];
    for (int i = 0; i < nv; ++i) {
        double s = 0.0;
        for (int64_t r = blockIdx.x * (int64_t)kBlock + threadIdx.x; r < n;
             r += (int64_t)gridDim.x * kBlock)
            s += M[(int64_t)i * n + r] * w[r];
        s = block_sum(s, sh);
        if (threadIdx.x == 0) part[(int64_t)i * kRedBlocks + blockIdx.x] = s;
    }
}

// out[i] = sum of part[i * kRedBlocks + 0 .. nparts) in block order (one CTA per vector).
__global__ void k_fold_many(const double* __restrict__ part, int nparts, double* __restrict__ out) {
    __shared__ double sh[kBlock / 32];
    double s = 0.0;
    for (int j = threadIdx.x; j < nparts; j += kBlock) s += part[(int64_t)blockIdx.x * kRedBlocks + j];
    s = block_sum(s, sh);
    if (threadIdx.x == 0) out[blockIdx.x] = s;
}

// w -= V c over vectors 0..nv-1.
__global__ void k_orth_update(int64_t n, int nv, const double* __restrict__ V,
                              const double* __restrict__ c, double* __restrict__ w) {
    for (int64_t i = blockIdx.x * (int64_t)kBlock + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * kBlock) {
        double a = w[i];
        for (int j = 0; j < nv; ++j) a -= c[j] * V[(int64_t)j * n + i];
        w[i] = a;
    }
}

// y = (x - a u - b up) (up may be null)
__global__ void k_three_term(int64_t n, const double* __restrict__ x, const double* __restrict__ u,
                             const double* __restrict__ up, const double* __restrict__ ab,
                             double* __restrict__ y) {
    const double a = ab[0], b = ab[1];
    for (int64_t i = blockIdx.x * (int64_t)kBlock + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * kBlock)
        y[i] = x[i] - a * u[i] - (up ? b * up[i] : 0.0);
}

__global__ void k_scale2(int64_t n, const double* __restrict__ s, const double* __restrict__ a,
                         const double* __restrict__ b, double* __restrict__ ya,
                         double* __restrict__ yb) {
    const double f = 1.0 / s[0];
    for (int64_t i = blockIdx.x * (int64_t)kBlock + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * kBlock) {
        ya[i] = a[i] * f;
        yb[i] = b[i] * f;
    }
}

// y = x - x[root] per component (out of place): every Lanczos vector is grounded at its
// component's representative, so no null-space component can build up.
__global__ void k_ground(int64_t n, const int32_t* __restrict__ root, const double* __restrict__ x,
                         double* __restrict__ y) {
    for (int64_t i = blockIdx.x * (int64_t)kBlock + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * kBlock)
        y[i] = x[i] - x[root[i]];
}

__global__ void k_complement(int64_t m, const uint8_t* __restrict__ mask, uint8_t* __restrict__ q) {
    for (int64_t e = blockIdx.x * (int64_t)kBlock + threadIdx.x; e < m;
         e += (int64_t)gridDim.x * kBlock)
        q[e] = mask[e] ? 0 : 1;
}

__global__ void k_seed_vec(int64_t n, uint64_t seed, double* __restrict__ v) {
    const uint64_t s0 = sfg_splitmix64(seed);
    for (int64_t i = blockIdx.x * (int64_t)kBlock + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * kBlock)
        v[i] = (double)(sfg_splitmix64(s0 + (uint64_t)i) >> 11) * 0x1.0p-53 - 0.5;
}

// Extreme eigenvalues of the symmetric tridiagonal matrix (alpha[0..m), beta[1..m)) by bisection
// on Sturm counts; out[0] = smallest, out[1] = largest.
__global__ void k_tridiag_extremes(int m, const double* __restrict__ alpha,
                                   const double* __restrict__ beta, double* __restrict__ out) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double lo = alpha[0], hi = alpha[0];
    for (int i = 0; i < m; ++i) {  // Gershgorin
        const double r = (i > 0 ? fabs(beta[i]) : 0.0) + (i + 1 < m ? fabs(beta[i + 1]) : 0.0);
        lo = fmin(lo, alpha[i] - r);
        hi = fmax(hi, alpha[i] + r);
    }
    auto count_below = [&](double x) {  // eigenvalues < x
        int c = 0;
        double q = 1.0;
        for (int i = 0; i < m; ++i) {
            const double b2 = i > 0 ? beta[i] * beta[i] : 0.0;
            q = alpha[i] - x - (i > 0 ? b2 / q : 0.0);
            if (q == 0.0) q = -1e-300;
            if (q < 0.0) ++c;
        }
        return c;
    };
    for (int which = 0; which < 2; ++which) {
        double a = lo, b = hi;
        const int target = which == 0 ? 1 : m;  // the 1st / m-th smallest
        for (int it = 0; it < 200 && b - a > 1e-15 * fmax(fabs(a), fabs(b)); ++it) {
            const double mid = 0.5 * (a + b);
            if (count_below(mid) >= target) b = mid; else a = mid;
        }
        out[which] = 0.5 * (a + b);
    }
}

// ---------------------------------------------------------------- host orchestration ------------

struct Factor {
    int32_t n = 0;
    int rounds = 0;
    std::vector<int64_t> round_k;    // eliminations of round r: order[round_k[r], round_k[r+1])
    std::vector<int64_t> round_seg;  // forward segments of round r: [round_seg[r], round_seg[r+1])
    int32_t* order = nullptr;
    int32_t *nb0 = nullptr, *nb1 = nullptr;
    double *w0 = nullptr, *w1 = nullptr;
    int64_t* seg_start = nullptr;
    int32_t* seg_target = nullptr;
    uint32_t* cval = nullptr;
    int32_t* csrc = nullptr;
    double* ccoef = nullptr;
    int32_t nc = 0;                  // core
    int32_t* core_nodes = nullptr;
    int64_t* crp = nullptr;
    int32_t* ccol = nullptr;
    double *cw = nullptr, *cd = nullptr;
};

sfg_status factorise(sfg_ctx* ctx, Scratch& s, const sfg_graph* P, Factor& F) {
    const int32_t n = P->n;
    const int64_t m = P->m;
    F.n = n;
    Scratch t(ctx);  // factorisation-only scratch
    int32_t *adj, *eu, *ev;
    double* ew;
    uint8_t *ealive, *nalive, *cand, *chosen;
    int64_t* pos;
    SFG_TRY(t.get(&adj, 2 * m));
    SFG_TRY(t.get(&eu, m));
    SFG_TRY(t.get(&ev, m));
    SFG_TRY(t.get(&ew, m));
    SFG_TRY(t.get(&ealive, m));
    SFG_TRY(t.get(&nalive, n));
    SFG_TRY(t.get(&cand, n));
    SFG_TRY(t.get(&chosen, n));
    SFG_TRY(t.get(&pos, (size_t)n + 1));
    SFG_TRY(s.get(&F.order, n));
    SFG_TRY(s.get(&F.nb0, n));
    SFG_TRY(s.get(&F.nb1, n));
    SFG_TRY(s.get(&F.w0, n));
    SFG_TRY(s.get(&F.w1, n));
    uint64_t* ckey;
    uint32_t* cval;
    SFG_TRY(t.get(&ckey, 2 * (size_t)n));
    SFG_TRY(t.get(&cval, 2 * (size_t)n));
    SFG_TRY(s.get(&F.csrc, 2 * (size_t)n));
    SFG_TRY(s.get(&F.ccoef, 2 * (size_t)n));
    cudaStream_t st = ctx->stream;
    SFG_CUDA(ctx, cudaMemcpyAsync(adj, P->eid, sizeof(int32_t) * 2 * m, cudaMemcpyDeviceToDevice, st));
    SFG_CUDA(ctx, cudaMemcpyAsync(eu, P->eu, sizeof(int32_t) * m, cudaMemcpyDeviceToDevice, st));
    SFG_CUDA(ctx, cudaMemcpyAsync(ev, P->ev, sizeof(int32_t) * m, cudaMemcpyDeviceToDevice, st));
    SFG_CUDA(ctx, cudaMemsetAsync(ealive, 1, m, st));
    SFG_CUDA(ctx, cudaMemsetAsync(nalive, 1, n, st));
    SFG_CUDA(ctx, cudaMemsetAsync(ckey, 0xff, sizeof(uint64_t) * 2 * n, st));
    // FP64 working weights
    {
        const float* src = P->ew;
        double* dst = ew;
        const int64_t mm = m;
        k_widen<<<grid_of(ctx, k_widen, m), kBlock, 0, st>>>(mm, src, dst);
        ++ctx->launches;
        SFG_LAUNCH_CHECK(ctx, "k_widen");
    }
    const int gn = grid_of(ctx, k_el_scan, n);
    int64_t done = 0;
    F.round_k.assign(1, 0);
    for (int round = 0; round < kMaxRounds && done < n; ++round) {
        k_el_scan<<<gn, kBlock, 0, st>>>(n, P->row_ptr, adj, eu, ev, ew, ealive, nalive, cand,
                                          F.nb0, F.nb1, F.w0, F.w1);
        k_el_choose<<<gn, kBlock, 0, st>>>(n, round, cand, F.nb0, F.nb1, chosen);
        ctx->launches += 2;
        SFG_LAUNCH_CHECK(ctx, "k_el_scan");
        SFG_TRY(sfg_scan_u8(ctx, chosen, pos, n));
        int64_t cnt = 0;
        SFG_TRY(sfg_read_i64(ctx, pos + n, &cnt));
        if (cnt == 0) break;
        k_el_apply<<<gn, kBlock, 0, st>>>(n, round, chosen, pos, done, P->row_ptr, adj, eu, ev, ew,
                                           ealive, nalive, F.nb0, F.nb1, F.w0, F.w1, F.order, ckey,
                                           cval, F.csrc, F.ccoef);
        ++ctx->launches;
        SFG_LAUNCH_CHECK(ctx, "k_el_apply");
        done += cnt;
        F.round_k.push_back(done);
        F.rounds = round + 1;
    }
    // contributions sorted by (round, target), entry order kept within a target
    const int64_t len = 2 * done;
    F.round_seg.assign(F.rounds + 1, 0);
    int64_t nseg = 0;
    if (len > 0) {
        uint64_t* kalt;
        uint32_t* valt;
        SFG_TRY(t.get(&kalt, len));
        SFG_TRY(t.get(&valt, len));
        SFG_TRY(sfg_radix_sort_pairs(ctx, &ckey, &cval, &kalt, &valt, len, 48));
        uint8_t* head;
        int64_t* hpos;
        SFG_TRY(t.get(&head, len));
        SFG_TRY(t.get(&hpos, len + 1));
        const int gl = grid_of(ctx, k_el_heads, len);
        k_el_heads<<<gl, kBlock, 0, st>>>(len, ckey, head);
        ++ctx->launches;
        SFG_LAUNCH_CHECK(ctx, "k_el_heads");
        SFG_TRY(sfg_scan_u8(ctx, head, hpos, len));
        SFG_TRY(sfg_read_i64(ctx, hpos + len, &nseg));
        int32_t* seg_round;
        SFG_TRY(s.get(&F.seg_start, nseg + 1));
        SFG_TRY(s.get(&F.seg_target, nseg + 1));
        SFG_TRY(t.get(&seg_round, nseg + 1));
        SFG_TRY(s.get(&F.cval, len));
        k_el_segs<<<gl, kBlock, 0, st>>>(len, ckey, head, hpos, F.seg_start, seg_round, F.seg_target);
        ++ctx->launches;
        SFG_LAUNCH_CHECK(ctx, "k_el_segs");
        // end of the last segment: the first unused key (keys of ~0 sort last)
        int64_t valid = 0;
        {
            int64_t* vcount;
            SFG_TRY(t.get(&vcount, 1));
            k_count_valid<<<1, kBlock, 0, st>>>(len, ckey, vcount);
            ++ctx->launches;
            SFG_LAUNCH_CHECK(ctx, "k_count_valid");
            SFG_TRY(sfg_read_i64(ctx, vcount, &valid));
        }
        SFG_CUDA(ctx, cudaMemcpyAsync(F.seg_start + nseg, &valid, sizeof(int64_t),
                                      cudaMemcpyHostToDevice, st));
        SFG_CUDA(ctx, cudaMemcpyAsync(F.cval, cval, sizeof(uint32_t) * len, cudaMemcpyDeviceToDevice, st));
        std::vector<int32_t> sr(nseg);
        if (nseg > 0)
            SFG_CUDA(ctx, cudaMemcpyAsync(sr.data(), seg_round, sizeof(int32_t) * nseg,
                                          cudaMemcpyDeviceToHost, st));
        SFG_CUDA(ctx, cudaStreamSynchronize(st));
        int64_t i = 0;
        for (int r = 0; r < F.rounds; ++r) {
            F.round_seg[r] = i;
            while (i < nseg && sr[i] == r) ++i;
        }
        F.round_seg[F.rounds] = i;
    }
    // the core
    int64_t* cid;
    SFG_TRY(t.get(&cid, (size_t)n + 1));
    k_core_flag<<<gn, kBlock, 0, st>>>(n, nalive, chosen);
    ++ctx->launches;
    SFG_TRY(sfg_scan_u8(ctx, chosen, cid, n));
    int64_t nc = 0;
    SFG_TRY(sfg_read_i64(ctx, cid + n, &nc));
    F.nc = (int32_t)nc;
    if (nc == 0) return SFG_OK;
    SFG_TRY(s.get(&F.core_nodes, nc));
    k_core_nodes<<<gn, kBlock, 0, st>>>(n, nalive, cid, F.core_nodes);
    ++ctx->launches;
    int64_t* epos;
    SFG_TRY(t.get(&epos, (size_t)m + 1));
    SFG_TRY(sfg_scan_u8(ctx, ealive, epos, m));
    int64_t mc = 0;
    SFG_TRY(sfg_read_i64(ctx, epos + m, &mc));
    SFG_TRY(s.get(&F.crp, nc + 1));
    SFG_TRY(s.get(&F.cd, nc));
    const int64_t lc = 2 * mc;
    SFG_TRY(s.get(&F.ccol, lc));
    SFG_TRY(s.get(&F.cw, lc));
    if (lc > 0) {
        uint64_t *k1, *k2;
        uint32_t *v1, *v2;
        SFG_TRY(t.get(&k1, lc));
        SFG_TRY(t.get(&k2, lc));
        SFG_TRY(t.get(&v1, lc));
        SFG_TRY(t.get(&v2, lc));
        k_core_entries<<<grid_of(ctx, k_core_entries, m), kBlock, 0, st>>>(m, eu, ev, ealive, cid,
                                                                           epos, k1, v1);
        ++ctx->launches;
        SFG_LAUNCH_CHECK(ctx, "k_core_entries");
        SFG_TRY(sfg_radix_sort_pairs(ctx, &k1, &v1, &k2, &v2, lc, 64));
        k_core_csr<<<grid_of(ctx, k_core_csr, lc), kBlock, 0, st>>>(lc, F.nc, k1, v1, ew, F.crp,
                                                                    F.ccol, F.cw);
        ++ctx->launches;
        SFG_LAUNCH_CHECK(ctx, "k_core_csr");
    } else {
        SFG_CUDA(ctx, cudaMemsetAsync(F.crp, 0, sizeof(int64_t) * (nc + 1), st));
    }
    k_core_diag<<<grid_of(ctx, k_core_diag, nc), kBlock, 0, st>>>(F.nc, F.crp, F.cw, F.cd);
    ++ctx->launches;
    SFG_LAUNCH_CHECK(ctx, "k_core_diag");
    return SFG_OK;
}

struct Solver {
    sfg_ctx* ctx;
    const Factor& F;
    double *b, *bc, *xc, *r, *p, *q, *z, *part, *sc;
    int64_t cg_iters = 0;
    int cg_max = 0;

    Solver(sfg_ctx* c, const Factor& f) : ctx(c), F(f) {}

    sfg_status init(Scratch& s) {
        SFG_TRY(s.get(&b, F.n));
        const size_t nc = F.nc > 0 ? F.nc : 1;
        SFG_TRY(s.get(&bc, nc));
        SFG_TRY(s.get(&xc, nc));
        SFG_TRY(s.get(&r, nc));
        SFG_TRY(s.get(&p, nc));
        SFG_TRY(s.get(&q, nc));
        SFG_TRY(s.get(&z, nc));
        SFG_TRY(s.get(&part, 2 * kRedBlocks));
        SFG_TRY(s.get(&sc, 8));
        cg_max = (int)std::min<int64_t>(20 * (int64_t)F.nc + 200, 200000);
        return SFG_OK;
    }

    // x = L_P^+ rhs up to per-component constants (rhs is not modified).
    sfg_status solve(const double* rhs, double* x) {
        cudaStream_t st = ctx->stream;
        SFG_CUDA(ctx, cudaMemcpyAsync(b, rhs, sizeof(double) * F.n, cudaMemcpyDeviceToDevice, st));
        if (F.nc > 0) {  // |rhs|^2 -> sc[5]: the core CG stops relative to the whole right-hand side
            const int gd = std::min(kRedBlocks, grid_of(ctx, k_multidot, F.n));
            k_multidot<<<gd, kBlock, 0, st>>>(F.n, 1, rhs, rhs, part);
            k_fold_many<<<1, kBlock, 0, st>>>(part, gd, sc + 5);
            ctx->launches += 2;
        }
        for (int rd = 0; rd < F.rounds; ++rd) {
            const int64_t s0 = F.round_seg[rd], s1 = F.round_seg[rd + 1];
            if (s1 > s0) {
                k_sv_forward<<<grid_of(ctx, k_sv_forward, s1 - s0), kBlock, 0, st>>>(
                    s0, s1, F.seg_start, F.seg_target, F.cval, F.csrc, F.ccoef, b);
                ++ctx->launches;
            }
        }
        SFG_LAUNCH_CHECK(ctx, "k_sv_forward");
        if (F.nc > 0) SFG_TRY(core_cg(x));
        for (int rd = F.rounds - 1; rd >= 0; --rd) {
            const int64_t k0 = F.round_k[rd], k1 = F.round_k[rd + 1];
            k_sv_backward<<<grid_of(ctx, k_sv_backward, k1 - k0), kBlock, 0, st>>>(
                k0, k1, F.order, F.nb0, F.nb1, F.w0, F.w1, b, x);
            ++ctx->launches;
        }
        SFG_LAUNCH_CHECK(ctx, "k_sv_backward");
        return SFG_OK;
    }

    sfg_status core_cg(double* x) {
        cudaStream_t st = ctx->stream;
        const int32_t nc = F.nc;
        const int gc = std::min(kRedBlocks, grid_of(ctx, k_cg_spmv, nc));
        k_gather<<<grid_of(ctx, k_gather, nc), kBlock, 0, st>>>(nc, F.core_nodes, b, bc);
        k_cg_init<<<gc, kBlock, 0, st>>>(nc, bc, F.cd, xc, r, p, part);
        k_cg_fold<<<1, kBlock, 0, st>>>(part, gc, 0, sc);
        ctx->launches += 3;
        SFG_LAUNCH_CHECK(ctx, "k_cg_init");
        double h[8];
        SFG_CUDA(ctx, cudaMemcpyAsync(h, sc, sizeof(double) * 8, cudaMemcpyDeviceToHost, st));
        SFG_CUDA(ctx, cudaStreamSynchronize(st));
        bool ok = h[7] != 0.0;
        for (int it = 0; !ok && it < cg_max;) {
            for (int k = 0; k < 16; ++k, ++it) {
                k_cg_spmv<<<gc, kBlock, 0, st>>>(nc, F.crp, F.ccol, F.cw, F.cd, p, q, part, sc);
                k_cg_fold<<<1, kBlock, 0, st>>>(part, gc, 1, sc);
                k_cg_update<<<gc, kBlock, 0, st>>>(nc, sc, F.cd, p, q, xc, r, z, part);
                k_cg_fold<<<1, kBlock, 0, st>>>(part, gc, 2, sc);
                k_cg_dir<<<gc, kBlock, 0, st>>>(nc, sc, z, p);
                ctx->launches += 5;
            }
            SFG_LAUNCH_CHECK(ctx, "core CG");
            SFG_CUDA(ctx, cudaMemcpyAsync(h, sc, sizeof(double) * 8, cudaMemcpyDeviceToHost, st));
            SFG_CUDA(ctx, cudaStreamSynchronize(st));
            cg_iters += 16;
            ok = h[7] != 0.0 && h[3] == h[3];
            if (h[7] != 0.0) break;
        }
        if (!ok)
            return sfg_fail(ctx, SFG_ETIMEOUT, "sfg_kappa: core CG did not converge in %d iterations",
                            cg_max);
        k_scatter<<<grid_of(ctx, k_scatter, nc), kBlock, 0, st>>>(nc, F.core_nodes, xc, x);
        ++ctx->launches;
        SFG_LAUNCH_CHECK(ctx, "k_scatter");
        return SFG_OK;
    }
};



// Per-component means in a fixed order: nodes sorted by (component label, id); small components
// are summed by one thread each in that order, large ones by one CTA each with a fixed
// assignment and tree (deterministic either way).
__global__ void k_comp_keys(int32_t n, const int32_t* __restrict__ root, uint64_t* __restrict__ key,
                            uint32_t* __restrict__ val) {
    for (int64_t v = blockIdx.x * (int64_t)kBlock + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * kBlock) {
        key[v] = ((uint64_t)(uint32_t)root[v] << 32) | (uint32_t)v;
        val[v] = (uint32_t)v;
    }
}

__global__ void k_comp_heads(int32_t n, const uint64_t* __restrict__ key, uint8_t* __restrict__ head) {
    for (int64_t i = blockIdx.x * (int64_t)kBlock + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * kBlock)
        head[i] = i == 0 || (key[i] >> 32) != (key[i - 1] >> 32);
}

__global__ void k_comp_segs(int32_t n, const uint64_t* __restrict__ key, const uint8_t* __restrict__ head,
                            const int64_t* __restrict__ hpos, int64_t* __restrict__ seg_start) {
    for (int64_t i = blockIdx.x * (int64_t)kBlock + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * kBlock)
        if (head[i]) seg_start[hpos[i]] = i;
}

constexpr int64_t kBigSeg = 2048;  // components at least this large get one CTA each

// Small components: one thread each, members summed in order.
__global__ void k_comp_mean(int64_t nseg, const int64_t* __restrict__ seg_start,
                            const uint32_t* __restrict__ order, const int32_t* __restrict__ root,
                            const double* __restrict__ x, double* __restrict__ mean_by_root) {
    for (int64_t s = blockIdx.x * (int64_t)kBlock + threadIdx.x; s < nseg;
         s += (int64_t)gridDim.x * kBlock) {
        const int64_t a = seg_start[s], b = seg_start[s + 1];
        if (b - a >= kBigSeg) continue;
        double acc = 0.0;
        for (int64_t i = a; i < b; ++i) acc += x[order[i]];
        mean_by_root[root[order[a]]] = acc / (double)(b - a);
    }
}

// Large components: one CTA each, a fixed thread-stride assignment and a fixed-shape tree.
__global__ void k_comp_mean_big(const int64_t* __restrict__ big, const int64_t* __restrict__ seg_start,
                                const uint32_t* __restrict__ order, const int32_t* __restrict__ root,
                                const double* __restrict__ x, double* __restrict__ mean_by_root) {
    __shared__ double sh[kBlock / 32];
    const int64_t s = big[blockIdx.x];
    const int64_t a = seg_start[s], b = seg_start[s + 1];
    double acc = 0.0;
    for (int64_t i = a + threadIdx.x; i < b; i += kBlock) acc += x[order[i]];
    acc = block_sum(acc, sh);
    if (threadIdx.x == 0) mean_by_root[root[order[a]]] = acc / (double)(b - a);
}

__global__ void k_sub_mean(int32_t n, const int32_t* __restrict__ root,
                           const double* __restrict__ mean_by_root, double* __restrict__ x) {
    for (int64_t v = blockIdx.x * (int64_t)kBlock + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * kBlock)
        x[v] -= mean_by_root[root[v]];
}

__global__ void k_pcg_update(int64_t n, double alpha, const double* __restrict__ p,
                             const double* __restrict__ q, double* __restrict__ x,
                             double* __restrict__ r) {
    for (int64_t i = blockIdx.x * (int64_t)kBlock + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * kBlock) {
        x[i] += alpha * p[i];
        r[i] -= alpha * q[i];
    }
}

__global__ void k_pcg_dir(int64_t n, double beta, const double* __restrict__ z, double* __restrict__ p) {
    for (int64_t i = blockIdx.x * (int64_t)kBlock + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * kBlock)
        p[i] = z[i] + beta * p[i];
}

// Diagonal preconditioner (the baseline): z = r / d, 0 where d = 0.
__global__ void k_pcg_diag(int32_t n, const double* __restrict__ deg, const double* __restrict__ r,
                           double* __restrict__ z) {
    for (int64_t i = blockIdx.x * (int64_t)kBlock + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * kBlock)
        z[i] = deg[i] > 0.0 ? r[i] / deg[i] : 0.0;
}

struct GraphGuard {
    sfg_graph* g = nullptr;
    ~GraphGuard() { sfg_graph_free(g); }
};

__global__ void k_sqrt_beta(double* __restrict__ sc) {
    if (threadIdx.x == 0) sc[1] = sqrt(fmax(sc[2], 0.0));
}

sfg_status kappa_impl(sfg_ctx* ctx, const sfg_graph* G, const uint8_t* mask, int steps,
                      uint64_t seed, double* kappa, double* lam) {
    const int32_t n = G->n;
    cudaStream_t st = ctx->stream;
    if (n <= 1 || G->m == 0) {
        *kappa = 1.0;
        lam[0] = lam[1] = 1.0;
        return SFG_OK;
    }
    GraphGuard P;
    SFG_TRY(sfg_subgraph_impl(ctx, G, mask, &P.g));
    Scratch s(ctx);
    int32_t* root = nullptr;
    bool lmin_exact = false;
    int64_t kdim = 0;  // dimension of the Krylov space: n minus the components of G
    {  // P must span every component of G, else kappa is infinite
        uint8_t* tm;
        SFG_TRY(s.get(&tm, G->m));
        SFG_TRY(s.get(&root, n));
        int64_t tg = 0, tp = 0;
        SFG_TRY(sfg_mst_impl(ctx, G, nullptr, tm, &tg, root));
        SFG_TRY(sfg_mst_impl(ctx, P.g, nullptr, tm, &tp));
        if (tp < tg) {
            *kappa = INFINITY;
            lam[0] = 0.0;
            lam[1] = INFINITY;
            return SFG_OK;
        }
        const int64_t dim = (int64_t)n - ((int64_t)n - tg);  // complement of the null space
        kdim = dim;
        if (steps > dim) steps = (int)dim;
        // lambda_min = 1 exactly when Q = G \ P has more components than G: L_G = L_P + L_Q >= L_P,
        // and a vector constant on the components of Q but not on those of G has L_G x = L_P x
        // with L_P x != 0
        uint8_t* qmask;
        SFG_TRY(s.get(&qmask, G->m));
        k_complement<<<grid_of(ctx, k_complement, G->m), kBlock, 0, st>>>(G->m, mask, qmask);
        ++ctx->launches;
        SFG_LAUNCH_CHECK(ctx, "k_complement");
        GraphGuard Q;
        SFG_TRY(sfg_subgraph_impl(ctx, G, qmask, &Q.g));
        int64_t tq = 0;
        SFG_TRY(sfg_mst_impl(ctx, Q.g, nullptr, tm, &tq));
        lmin_exact = tq < tg;
    }
    Factor F;
    SFG_TRY(factorise(ctx, s, P.g, F));
    Solver S(ctx, F);
    SFG_TRY(S.init(s));
    const int m = steps;
    double *V, *U, *z, *w, *r, *part, *c, *sc, *dal, *dbe, *ext, *tmp;
    SFG_TRY(s.get(&V, (size_t)(m + 1) * n));
    SFG_TRY(s.get(&U, (size_t)(m + 1) * n));
    SFG_TRY(s.get(&z, n));
    SFG_TRY(s.get(&w, n));
    SFG_TRY(s.get(&r, n));
    SFG_TRY(s.get(&part, (size_t)(m + 1) * kRedBlocks));
    SFG_TRY(s.get(&c, m + 1));
    SFG_TRY(s.get(&sc, 8));
    SFG_TRY(s.get(&dal, m + 1));
    SFG_TRY(s.get(&dbe, m + 1));
    SFG_TRY(s.get(&ext, 2));
    SFG_TRY(s.get(&tmp, n));
    const int gv = grid_of(ctx, k_lap_mul, n);
    const int gd = std::min(kRedBlocks, grid_of(ctx, k_multidot, n));
    auto dot = [&](const double* a, const double* b, double* out) -> sfg_status {
        k_multidot<<<gd, kBlock, 0, st>>>(n, 1, a, b, part);
        k_fold_many<<<1, kBlock, 0, st>>>(part, gd, out);
        ctx->launches += 2;
        SFG_LAUNCH_CHECK(ctx, "dot");
        return SFG_OK;
    };
    auto rd = [&](double* h, const double* d, int k) -> sfg_status {
        SFG_CUDA(ctx, cudaMemcpyAsync(h, d, sizeof(double) * k, cudaMemcpyDeviceToHost, st));
        SFG_CUDA(ctx, cudaStreamSynchronize(st));
        return SFG_OK;
    };
    // v0: seeded, u0 = L_P v0, both scaled to unit L_P-norm
    k_seed_vec<<<gv, kBlock, 0, st>>>(n, seed, tmp);
    k_ground<<<gv, kBlock, 0, st>>>(n, root, tmp, w);
    k_lap_mul<<<gv, kBlock, 0, st>>>(n, P.g->row_ptr, P.g->colval, P.g->deg, w, r);
    ctx->launches += 3;
    SFG_TRY(dot(w, r, sc + 2));
    k_sqrt_beta<<<1, 32, 0, st>>>(sc);
    k_scale2<<<gv, kBlock, 0, st>>>(n, sc + 1, w, r, V, U);
    ctx->launches += 2;
    SFG_CUDA(ctx, cudaMemsetAsync(sc + 1, 0, sizeof(double), st));  // beta_0 = 0
    std::vector<double> alpha, beta(1, 0.0);
    double amax = 0.0;
    bool stop_cg = false;
    for (int j = 0; j < m; ++j) {
        double* vj = V + (size_t)j * n;
        double* uj = U + (size_t)j * n;
        k_lap_mul<<<gv, kBlock, 0, st>>>(n, G->row_ptr, G->colval, G->deg, vj, z);
        ++ctx->launches;
        SFG_TRY(dot(vj, z, sc + 0));
        k_three_term<<<gv, kBlock, 0, st>>>(n, z, uj, j > 0 ? uj - n : nullptr, sc, r);
        ++ctx->launches;
        SFG_LAUNCH_CHECK(ctx, "k_three_term");
        SFG_TRY(dot(r, r, sc + 3));
        SFG_TRY(dot(z, z, sc + 4));
        {  // r vanishing against L_G v_j: v_j spans an invariant subspace (e.g. P = G)
            double h[5];
            SFG_TRY(rd(h, sc, 5));
            if (!(h[3] > 1e-24 * h[4])) {
                alpha.push_back(h[0]);
                break;
            }
        }
        {
            const sfg_status ss = S.solve(r, tmp);
            // A core CG that does not converge once the Krylov space has run out (v_j is rounding
            // noise: an inconsistent right-hand side) marks a breakdown, and T_j (without this
            // step) holds the Ritz values. That can only happen late, after at least half of the
            // Krylov dimension; an earlier failure (a core too ill-conditioned for CG to reach
            // the tolerance) is reported as an error instead of a kappa from a truncated space.
            if (ss == SFG_ETIMEOUT && j > 0 && 2 * (int64_t)(j + 1) >= kdim) {
                stop_cg = true;
                break;
            }
            if (ss != SFG_OK) return ss;
        }
        k_ground<<<gv, kBlock, 0, st>>>(n, root, tmp, w);
        ++ctx->launches;
        for (int pass = 0; pass < 2; ++pass) {  // full reorthogonalisation in the L_P product
            k_multidot<<<gd, kBlock, 0, st>>>(n, j + 1, U, w, part);
            k_fold_many<<<j + 1, kBlock, 0, st>>>(part, gd, c);
            k_orth_update<<<gv, kBlock, 0, st>>>(n, j + 1, V, c, w);
            ctx->launches += 3;
            SFG_LAUNCH_CHECK(ctx, "reorthogonalisation");
        }
        // u_{j+1} from an explicit product: carried by the recurrence it drifts out of the range
        // of L_P and the next right-hand sides stop being consistent
        k_lap_mul<<<gv, kBlock, 0, st>>>(n, P.g->row_ptr, P.g->colval, P.g->deg, w, r);
        ++ctx->launches;
        SFG_TRY(dot(w, r, sc + 2));
        double h[3];
        SFG_TRY(rd(h, sc, 3));
        alpha.push_back(h[0]);
        amax = std::max(amax, std::fabs(h[0]));
        const double b2 = h[2];
        // breakdown: beta below 1e-10 of the largest |alpha| (the Krylov space is exhausted)
        if (!(b2 > 1e-20 * amax * amax) || j + 1 == m) break;
        beta.push_back(std::sqrt(b2));
        k_sqrt_beta<<<1, 32, 0, st>>>(sc);
        k_scale2<<<gv, kBlock, 0, st>>>(n, sc + 1, w, r, V + (size_t)(j + 1) * n,
                                        U + (size_t)(j + 1) * n);
        ctx->launches += 2;
        SFG_LAUNCH_CHECK(ctx, "k_scale2");
    }
    const int mm = (int)alpha.size();
    beta.resize(mm, 0.0);
    SFG_CUDA(ctx, cudaMemcpyAsync(dal, alpha.data(), sizeof(double) * mm, cudaMemcpyHostToDevice, st));
    SFG_CUDA(ctx, cudaMemcpyAsync(dbe, beta.data(), sizeof(double) * mm, cudaMemcpyHostToDevice, st));
    k_tridiag_extremes<<<1, 32, 0, st>>>(mm, dal, dbe, ext);
    ++ctx->launches;
    SFG_LAUNCH_CHECK(ctx, "k_tridiag_extremes");
    double e[2];
    SFG_TRY(rd(e, ext, 2));
    lam[0] = lmin_exact ? 1.0 : e[0];
    lam[1] = e[1];
    lam[2] = mm;
    lam[3] = (double)S.cg_iters;
    lam[4] = stop_cg ? 1.0 : 0.0;
    lam[5] = lmin_exact ? 1.0 : 0.0;
    *kappa = lam[1] / lam[0];
    return SFG_OK;
}

// Mean removal per component of G (labels = component representatives).
struct CompMean {
    int32_t n = 0;
    const int32_t* root = nullptr;
    uint32_t* order = nullptr;
    int64_t* seg_start = nullptr;
    int64_t nseg = 0;
    double* mean_by_root = nullptr;
    int64_t* big = nullptr;  // indices of the components with >= kBigSeg members
    int64_t nbig = 0;

    sfg_status init(sfg_ctx* ctx, Scratch& s, int32_t n_, const int32_t* root_) {
        n = n_;
        root = root_;
        cudaStream_t st = ctx->stream;
        Scratch t(ctx);
        uint64_t *k1, *k2;
        uint32_t* v2;
        uint8_t* head;
        int64_t* hpos;
        SFG_TRY(t.get(&k1, n));
        SFG_TRY(t.get(&k2, n));
        SFG_TRY(s.get(&order, n));
        SFG_TRY(t.get(&v2, n));
        SFG_TRY(t.get(&head, n));
        SFG_TRY(t.get(&hpos, (size_t)n + 1));
        SFG_TRY(s.get(&mean_by_root, n));
        k_comp_keys<<<grid_of(ctx, k_comp_keys, n), kBlock, 0, st>>>(n, root, k1, order);
        ++ctx->launches;
        uint32_t* const alt = v2;
        SFG_TRY(sfg_radix_sort_pairs(ctx, &k1, &order, &k2, &v2, n, 64));
        if (order == alt) {  // sorted values ended in the temporary buffer: keep it with s
            t.release(alt);
            s.ptrs.push_back(alt);
        }
        k_comp_heads<<<grid_of(ctx, k_comp_heads, n), kBlock, 0, st>>>(n, k1, head);
        ++ctx->launches;
        SFG_TRY(sfg_scan_u8(ctx, head, hpos, n));
        SFG_TRY(sfg_read_i64(ctx, hpos + n, &nseg));
        SFG_TRY(s.get(&seg_start, nseg + 1));
        k_comp_segs<<<grid_of(ctx, k_comp_segs, n), kBlock, 0, st>>>(n, k1, head, hpos, seg_start);
        ++ctx->launches;
        const int64_t nn = n;
        SFG_CUDA(ctx, cudaMemcpyAsync(seg_start + nseg, &nn, sizeof(int64_t), cudaMemcpyHostToDevice, st));
        std::vector<int64_t> hs(nseg + 1), hb;
        SFG_CUDA(ctx, cudaMemcpyAsync(hs.data(), seg_start, sizeof(int64_t) * (nseg + 1),
                                      cudaMemcpyDeviceToHost, st));
        SFG_CUDA(ctx, cudaStreamSynchronize(st));
        SFG_LAUNCH_CHECK(ctx, "component segments");
        for (int64_t i = 0; i < nseg; ++i)
            if (hs[i + 1] - hs[i] >= kBigSeg) hb.push_back(i);
        nbig = (int64_t)hb.size();
        if (nbig > 0) {
            SFG_TRY(s.get(&big, nbig));
            SFG_CUDA(ctx, cudaMemcpyAsync(big, hb.data(), sizeof(int64_t) * nbig,
                                          cudaMemcpyHostToDevice, st));
            SFG_CUDA(ctx, cudaStreamSynchronize(st));
        }
        return SFG_OK;
    }

    sfg_status remove(sfg_ctx* ctx, double* x) {
        k_comp_mean<<<grid_of(ctx, k_comp_mean, nseg), kBlock, 0, ctx->stream>>>(
            nseg, seg_start, order, root, x, mean_by_root);
        if (nbig > 0)
            k_comp_mean_big<<<(unsigned)nbig, kBlock, 0, ctx->stream>>>(big, seg_start, order, root,
                                                                        x, mean_by_root);
        k_sub_mean<<<grid_of(ctx, k_sub_mean, n), kBlock, 0, ctx->stream>>>(n, root, mean_by_root, x);
        ctx->launches += nbig > 0 ? 3 : 2;
        SFG_LAUNCH_CHECK(ctx, "component means");
        return SFG_OK;
    }
};

sfg_status pcg_impl(sfg_ctx* ctx, const sfg_graph* G, const uint8_t* mask, const double* b,
                    double tol, int maxit, double* x, int* iters, double* relres) {
    const int32_t n = G->n;
    cudaStream_t st = ctx->stream;
    *iters = 0;
    *relres = 0.0;
    if (n == 0) return SFG_OK;
    Scratch s(ctx);
    int32_t* root;
    uint8_t* tm;
    SFG_TRY(s.get(&root, n));
    SFG_TRY(s.get(&tm, G->m > 0 ? G->m : 1));
    int64_t tg = 0;
    SFG_TRY(sfg_mst_impl(ctx, G, nullptr, tm, &tg, root));
    GraphGuard P;
    Factor F;
    Solver* S = nullptr;
    struct Del { Solver** p; ~Del() { delete *p; } } del{&S};
    if (mask) {
        SFG_TRY(sfg_subgraph_impl(ctx, G, mask, &P.g));
        int64_t tp = 0;
        SFG_TRY(sfg_mst_impl(ctx, P.g, nullptr, tm, &tp));
        if (tp < tg) return sfg_fail(ctx, SFG_EINVAL, "sfg_solve_pcg: P does not span G's components");
        SFG_TRY(factorise(ctx, s, P.g, F));
        S = new Solver(ctx, F);
        SFG_TRY(S->init(s));
    }
    CompMean cm;
    SFG_TRY(cm.init(ctx, s, n, root));
    double *r, *z, *p, *q, *part, *sc;
    SFG_TRY(s.get(&r, n));
    SFG_TRY(s.get(&z, n));
    SFG_TRY(s.get(&p, n));
    SFG_TRY(s.get(&q, n));
    SFG_TRY(s.get(&part, kRedBlocks));
    SFG_TRY(s.get(&sc, 4));
    const int gv = grid_of(ctx, k_lap_mul, n);
    const int gd = std::min(kRedBlocks, grid_of(ctx, k_multidot, n));
    auto dot = [&](const double* a, const double* c, double* out_host) -> sfg_status {
        k_multidot<<<gd, kBlock, 0, st>>>(n, 1, a, c, part);
        k_fold_many<<<1, kBlock, 0, st>>>(part, gd, sc);
        ctx->launches += 2;
        SFG_LAUNCH_CHECK(ctx, "dot");
        SFG_CUDA(ctx, cudaMemcpyAsync(out_host, sc, sizeof(double), cudaMemcpyDeviceToHost, st));
        SFG_CUDA(ctx, cudaStreamSynchronize(st));
        return SFG_OK;
    };
    // The recursive residual drifts off range(L_G) by rounding while it shrinks, which would make
    // the core system inconsistent relative to its size: project it before every application.
    auto precond = [&](double* rr, double* zz) -> sfg_status {
        SFG_TRY(cm.remove(ctx, rr));
        if (S) {
            SFG_TRY(S->solve(rr, zz));
        } else {
            k_pcg_diag<<<gv, kBlock, 0, st>>>(n, G->deg, rr, zz);
            ++ctx->launches;
        }
        return cm.remove(ctx, zz);
    };
    // r = b projected onto range(L_G); x = 0
    SFG_CUDA(ctx, cudaMemcpyAsync(r, b, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
    SFG_TRY(cm.remove(ctx, r));
    SFG_CUDA(ctx, cudaMemsetAsync(x, 0, sizeof(double) * n, st));
    double bb = 0.0;
    SFG_TRY(dot(r, r, &bb));
    if (bb == 0.0) return SFG_OK;
    SFG_TRY(precond(r, z));
    SFG_CUDA(ctx, cudaMemcpyAsync(p, z, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
    double rz = 0.0, rr = bb;
    SFG_TRY(dot(r, z, &rz));
    int it = 0;
    while (it < maxit && rr > tol * tol * bb) {
        k_lap_mul<<<gv, kBlock, 0, st>>>(n, G->row_ptr, G->colval, G->deg, p, q);
        ++ctx->launches;
        double pq = 0.0;
        SFG_TRY(dot(p, q, &pq));
        if (!(pq > 0.0)) break;
        const double alpha = rz / pq;
        k_pcg_update<<<gv, kBlock, 0, st>>>(n, alpha, p, q, x, r);
        ++ctx->launches;
        ++it;
        SFG_TRY(dot(r, r, &rr));
        if (rr <= tol * tol * bb) break;
        SFG_TRY(precond(r, z));
        double rz2 = 0.0;
        SFG_TRY(dot(r, z, &rz2));
        k_pcg_dir<<<gv, kBlock, 0, st>>>(n, rz2 / rz, z, p);
        ++ctx->launches;
        rz = rz2;
    }
    SFG_TRY(cm.remove(ctx, x));
    *iters = it;
    *relres = std::sqrt(rr / bb);
    return SFG_OK;
}

}  // namespace

sfg_status sfg_kappa_impl(sfg_ctx* ctx, const sfg_graph* G, const uint8_t* mask, int steps,
                          uint64_t seed, double* kappa, double* info6) {
    double info[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    SFG_TRY(kappa_impl(ctx, G, mask, steps, seed, kappa, info));
    if (info6)
        for (int i = 0; i < 6; ++i) info6[i] = info[i];
    return SFG_OK;
}

extern "C" SFG_API sfg_status sfg_kappa(sfg_ctx* ctx, const sfg_graph* G, const uint8_t* mask,
                                        int steps, uint64_t seed, double* kappa_host,
                                        double* info_host) {
    if (!ctx) return SFG_EINVAL;
    SFG_DEVICE(ctx);
    if (!G || !kappa_host) return sfg_fail(ctx, SFG_EINVAL, "sfg_kappa: G and kappa_host are required");
    if (steps < 1) return sfg_fail(ctx, SFG_EINVAL, "sfg_kappa: steps must be >= 1");
    if (G->m > 0) SFG_TRY(sfg_check_dev(ctx, mask, "mask"));
    return sfg_kappa_impl(ctx, G, mask, steps, seed, kappa_host, info_host);
}

extern "C" SFG_API sfg_status sfg_solve_pcg(sfg_ctx* ctx, const sfg_graph* G, const uint8_t* mask,
                                            const double* b, double tol, int maxit, double* x,
                                            int* iters_host, double* relres_host) {
    if (!ctx) return SFG_EINVAL;
    SFG_DEVICE(ctx);
    if (!G) return sfg_fail(ctx, SFG_EINVAL, "graph is NULL");
    if (!(tol > 0.0) || maxit < 0) return sfg_fail(ctx, SFG_EINVAL, "tol must be > 0 and maxit >= 0");
    if (G->n > 0) {
        SFG_TRY(sfg_check_dev(ctx, b, "b"));
        SFG_TRY(sfg_check_dev(ctx, x, "x"));
    }
    if (mask && G->m > 0) SFG_TRY(sfg_check_dev(ctx, mask, "mask"));
    int it = 0;
    double rel = 0.0;
    SFG_TRY(pcg_impl(ctx, G, mask, b, tol, maxit, x, &it, &rel));
    if (iters_host) *iters_host = it;
    if (relres_host) *relres_host = rel;
    return SFG_OK;
}
