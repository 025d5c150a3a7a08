// kernels.cu -- sm_103a kernels of the state-vector hot path.
//
//   k_tile_pass     one pass of the fused program: each block gathers the
//                   2^m amplitudes of one tile (the non-tile qubits fixed by
//                   blockIdx) into shared memory, applies every op of the pass
//                   (Eq. (1q-op)/(2q-op) generalised to dense 2^k blocks on
//                   tile-local qubits), and writes the tile back.
//   k_resident      the whole state lives in one block's shared memory and the
//                   whole instruction stream -- dense ops, measurements, resets
//                   -- runs in one launch (one block per state for batches).
//   k_prob          FP64 Born probabilities of one qubit: per-block partials,
//                   then the last block to arrive sums them (a fixed-shape
//                   strided sum and warp tree), draws (or asserts) the
//                   outcome and writes the scale.
//   k_collapse      zero the rejected half, scale the kept half by
//                   1/sqrt(p_outcome) in FP64 (RESET: move |1> onto |0>).
//   k_expect        <psi|P_t|psi> partial sums in FP64 per (block, term),
//                   k_expect_final sums them in block order.
//
// State layout: 2^n interleaved (re, im) amplitudes, qubit q = index bit q.
// Every wait in this file is a __syncthreads; no kernel spins on memory.
#include "kernels.h"

#include <algorithm>
#include <cstdint>
#include <cstring>

namespace qsim {

namespace {

template <typename R> struct V2;
template <> struct V2<float> { using T = float2; };
template <> struct V2<double> { using T = double2; };

__device__ __forceinline__ float2 czero(float2) { return make_float2(0.f, 0.f); }
__device__ __forceinline__ double2 czero(double2) { return make_double2(0.0, 0.0); }

__device__ __forceinline__ void cmac(float2 &acc, const float2 m, const float2 x) {
    acc.x = fmaf(m.x, x.x, acc.x);
    acc.x = fmaf(-m.y, x.y, acc.x);
    acc.y = fmaf(m.x, x.y, acc.y);
    acc.y = fmaf(m.y, x.x, acc.y);
}
__device__ __forceinline__ void cmac(double2 &acc, const double2 m, const double2 x) {
    acc.x = fma(m.x, x.x, acc.x);
    acc.x = fma(-m.y, x.y, acc.x);
    acc.y = fma(m.x, x.y, acc.y);
    acc.y = fma(m.y, x.x, acc.y);
}
__device__ __forceinline__ double norm2(float2 a) {
    double x = a.x, y = a.y;
    return x * x + y * y;
}
__device__ __forceinline__ double norm2(double2 a) { return a.x * a.x + a.y * a.y; }
// |a|^2 as a term of an FP64 sum.  complex64: formed in FP32 (the amplitude's
// own precision, relative error <= 2^-23), then widened, so each term costs
// one FP64-pipe operation of the sum (GB300's FP64 rate is 1/60 of FP32's);
// complex128: in FP64.
__device__ __forceinline__ double norm2_term(float2 a) { return (double)fmaf(a.x, a.x, a.y * a.y); }
__device__ __forceinline__ double norm2_term(double2 a) { return norm2(a); }
// Re(i^ny conj(b) a) (-1)^neg as a term of an FP64 sum, formed in the
// amplitudes' precision as norm2_term is.
__device__ __forceinline__ double pauli_term(float2 a, float2 b, int ny, unsigned neg) {
    const float wr = fmaf(b.x, a.x, b.y * a.y), wi = fmaf(b.x, a.y, -(b.y * a.x));
    float v = ny == 0 ? wr : ny == 1 ? -wi : ny == 2 ? -wr : wi;
    v = __int_as_float(__float_as_int(v) ^ (neg << 31));
    return (double)v;
}
__device__ __forceinline__ double pauli_term(double2 a, double2 b, int ny, unsigned neg) {
    const double wr = b.x * a.x + b.y * a.y, wi = b.x * a.y - b.y * a.x;
    const double v = ny == 0 ? wr : ny == 1 ? -wi : ny == 2 ? -wr : wi;
    return __longlong_as_double(__double_as_longlong(v) ^ ((unsigned long long)neg << 63));
}
// w with its sign flipped when neg = 1, by integer operations on the sign bit
// (no floating-point instruction: on the FP64 pipe that would cost as much as
// the rotation's fused multiply-adds).
__device__ __forceinline__ float flip_sign(float w, unsigned neg) {
    return __int_as_float(__float_as_int(w) ^ (neg << 31));
}
__device__ __forceinline__ double flip_sign(double w, unsigned neg) {
    return __longlong_as_double(__double_as_longlong(w) ^ ((unsigned long long)neg << 63));
}
__device__ __forceinline__ float2 scale_by(float2 a, double s) {
    return make_float2((float)((double)a.x * s), (float)((double)a.y * s));
}
__device__ __forceinline__ double2 scale_by(double2 a, double s) {
    return make_double2(a.x * s, a.y * s);
}
__device__ __forceinline__ float fma_r(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double fma_r(double a, double b, double c) { return fma(a, b, c); }

__device__ __forceinline__ unsigned ins0(unsigned x, int p) {
    return ((x >> p) << (p + 1)) | (x & ((1u << p) - 1u));
}
__device__ __forceinline__ uint64_t ins0_64(uint64_t x, int p) {
    return ((x >> p) << (p + 1)) | (x & ((1ull << p) - 1ull));
}

// ------------------------------------------------------ Philox4x64-10 --
// Salmon et al., SC'11: 10 rounds of the 4x64 bijection with key schedule
// k += (W0, W1) between rounds.
__device__ __forceinline__ uint64_t philox_word0(uint64_t ctr0, uint64_t seed, uint64_t ctr1 = 0) {
    const uint64_t M0 = 0xD2E7470EE14C6C93ULL, M1 = 0xCA5A826395121157ULL;
    const uint64_t W0 = 0x9E3779B97F4A7C15ULL, W1 = 0xBB67AE8584CAA73BULL;
    uint64_t c0 = ctr0, c1 = ctr1, c2 = 0, c3 = 0, k0 = seed, k1 = 0;
#pragma unroll
    for (int r = 0; r < 10; r++) {
        if (r) {
            k0 += W0;
            k1 += W1;
        }
        const uint64_t hi0 = __umul64hi(M0, c0), lo0 = M0 * c0;
        const uint64_t hi1 = __umul64hi(M1, c2), lo1 = M1 * c2;
        const uint64_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
    }
    return c0;
}
__device__ __forceinline__ double draw_u01(uint64_t seed, uint64_t k) {
    return (double)(philox_word0(k, seed) >> 11) * (1.0 / 9007199254740992.0);
}

struct Decision {
    int outcome;
    int fail;
    double scale;
    double prob;
};

// Outcome rule of the measurement (draw or assertion) from the raw sums.
__device__ Decision decide(double s0, double s1, int mode, int reset, uint64_t seed,
                           uint64_t ordinal, double thr) {
    Decision d;
    const double tot = s0 + s1;
    const double P0 = s0 / tot;
    d.fail = 0;
    if ((mode & 1) && !reset) {
        if (!(P0 > thr)) {
            d.fail = 1;
            d.outcome = -1;
            d.prob = P0;
            d.scale = 1.0;
            return d;
        }
        d.outcome = 0;
    } else {
        const double u = draw_u01(seed, ordinal);
        d.outcome = (u < P0) ? 0 : 1;
    }
    const double p_out = d.outcome ? s1 : s0;
    d.scale = 1.0 / sqrt(p_out);
    d.prob = d.outcome ? s1 / tot : P0;
    return d;
}

// Fixed-shape block reduction of two doubles (deterministic order).
template <int NT>
__device__ __forceinline__ void block_sum2(double &a, double &b, double *red /* 2*NT/32 */) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        b += __shfl_xor_sync(0xffffffffu, b, o);
    }
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) {
        red[2 * w] = a;
        red[2 * w + 1] = b;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double x = 0, y = 0;
        for (int i = 0; i < NT / 32; i++) {
            x += red[2 * i];
            y += red[2 * i + 1];
        }
        red[0] = x;
        red[1] = y;
    }
    __syncthreads();
    a = red[0];
    b = red[1];
    __syncthreads();
}

// ------------------------------------------------------------ dense ops --
// Amplitude offsets of the 2^K members of a group (bit j of the local matrix
// index <-> tile position lq[j]) and the positions sorted for zero insertion.
template <int K>
__device__ __forceinline__ void group_layout(const DevOp &op, int *sp, unsigned *off) {
#pragma unroll
    for (int j = 0; j < K; j++) sp[j] = op.lq[j];
#pragma unroll
    for (int i = 1; i < K; i++)
#pragma unroll
        for (int j = i; j > 0; j--)
            if (sp[j - 1] > sp[j]) {
                int t = sp[j - 1];
                sp[j - 1] = sp[j];
                sp[j] = t;
            }
#pragma unroll
    for (int l = 0; l < (1 << K); l++) {
        unsigned o = 0;
#pragma unroll
        for (int j = 0; j < K; j++) o |= ((unsigned)(l >> j) & 1u) << op.lq[j];
        off[l] = o;
    }
}

// K <= 2 (the paper's C1 / C2): the matrix lives in registers.
template <int K, typename T, int NT>
__device__ __forceinline__ void apply_dense_reg(T *tile, int m, const DevOp &op, const T *mats) {
    constexpr int D = 1 << K;
    int sp[K];
    unsigned off[D];
    group_layout<K>(op, sp, off);
    const T *M = mats + op.mat;
    T mr[D * D];
#pragma unroll
    for (int i = 0; i < D * D; i++) mr[i] = M[i];
    // U groups per thread per iteration, loaded before any is stored (groups
    // are disjoint), so shared-memory latency overlaps across them
    constexpr int U = K == 1 ? 4 : 2;
    const unsigned G = 1u << (m - K);
    for (unsigned g0 = threadIdx.x; g0 < G; g0 += U * NT) {
        unsigned bb[U];
        T x[U][D];
#pragma unroll
        for (int u = 0; u < U; u++) {
            const unsigned g = g0 + u * NT;
            unsigned b = g < G ? g : 0;
#pragma unroll
            for (int j = 0; j < K; j++) b = ins0(b, sp[j]);
            bb[u] = b;
#pragma unroll
            for (int l = 0; l < D; l++) x[u][l] = tile[b + off[l]];
        }
#pragma unroll
        for (int u = 0; u < U; u++) {
            if (g0 + u * NT >= G) break;
#pragma unroll
            for (int r = 0; r < D; r++) {
                T acc = czero(x[u][0]);
#pragma unroll
                for (int c = 0; c < D; c++) cmac(acc, mr[r * D + c], x[u][c]);
                tile[bb[u] + off[r]] = acc;
            }
        }
    }
}

// Monomial K-qubit op (K <= 2, see kMono1/kMono2): one complex multiply per
// amplitude.  The product is formed with the same fused multiply-adds, in the
// same order, as the nonzero term of apply_dense_reg's row sum (the zero terms
// there add exact zeros), so both give the same values.
template <int K, typename T, int NT>
__device__ __forceinline__ void apply_mono(T *tile, int m, const DevOp &op, const T *mats) {
    constexpr int D = 1 << K;
    int sp[K];
    unsigned off[D];
    group_layout<K>(op, sp, off);
    const T *M = mats + op.mat;
    T mr[D];
    unsigned offp[D];  // offset of the input each output row takes
#pragma unroll
    for (int r = 0; r < D; r++) {
        const int c = (op.flags >> (2 * r)) & (D - 1);
        mr[r] = M[r * D + c];
        unsigned o = 0;
#pragma unroll
        for (int j = 0; j < K; j++) o |= ((unsigned)(c >> j) & 1u) << op.lq[j];
        offp[r] = o;
    }
    constexpr int U = 4;
    const unsigned G = 1u << (m - K);
    for (unsigned g0 = threadIdx.x; g0 < G; g0 += U * NT) {
        unsigned bb[U];
        T x[U][D];
#pragma unroll
        for (int u = 0; u < U; u++) {
            const unsigned g = g0 + u * NT;
            unsigned b = g < G ? g : 0;
#pragma unroll
            for (int j = 0; j < K; j++) b = ins0(b, sp[j]);
            bb[u] = b;
#pragma unroll
            for (int r = 0; r < D; r++) x[u][r] = tile[b + offp[r]];
        }
#pragma unroll
        for (int u = 0; u < U; u++) {
            if (g0 + u * NT >= G) break;
#pragma unroll
            for (int r = 0; r < D; r++) {
                T acc = czero(x[u][0]);
                cmac(acc, mr[r], x[u][r]);
                tile[bb[u] + off[r]] = acc;
            }
        }
    }
}

// K >= 3: the matrix is read from shared memory (broadcast reads), so that its
// 4^K entries are not all held in registers.  STAGE: copy it from global into
// mbuf first; otherwise `mats` already points into shared memory.
template <int K, typename T, int NT, bool STAGE>
__device__ __forceinline__ void apply_dense_smem(T *tile, int m, const DevOp &op, const T *mats,
                                                 T *mbuf) {
    constexpr int D = 1 << K;
    const T *M = mats + op.mat;
    if constexpr (STAGE) {
        for (int i = threadIdx.x; i < D * D; i += NT) mbuf[i] = M[i];
        __syncthreads();
    } else {
        mbuf = const_cast<T *>(M);
    }
    int sp[K];
    unsigned off[D];
    group_layout<K>(op, sp, off);
    const unsigned G = 1u << (m - K);
    for (unsigned g = threadIdx.x; g < G; g += NT) {
        unsigned b = g;
#pragma unroll
        for (int j = 0; j < K; j++) b = ins0(b, sp[j]);
        T x[D];
#pragma unroll
        for (int l = 0; l < D; l++) x[l] = tile[b + off[l]];
        // every input is in registers before the first output is stored
#pragma unroll 1
        for (int r = 0; r < D; r++) {
            T acc = czero(x[0]);
            const T *row = mbuf + r * D;
#pragma unroll
            for (int c = 0; c < D; c++) cmac(acc, row[c], x[c]);
            unsigned o = 0;
#pragma unroll
            for (int j = 0; j < K; j++) o |= ((unsigned)(r >> j) & 1u) << op.lq[j];
            tile[b + o] = acc;
        }
    }
}

// Pauli rotation in tile coordinates (encoding in kernels.h): with x, z the
// tile-local X and Z masks, b = parity(zc & tile index), u = +-W,
//   a'_j = cos a_j + W (odd ? i : 1) (-1)^{parity(k & z) ^ b} a_k,   k = j ^ x.
// With x = 0 it is diagonal: a'_j = (cos + W (odd ? i : 1) (-1)^{parity(j & z) ^ b}) a_j.
// (c, w) pair update r = c a + u (odd ? i : 1) b, or in the scaled form (c = 1)
// r = a + u (odd ? i : 1) b, one fused multiply-add per component.  SCALED and
// ODD are compile-time, so each pair loop holds only its own arithmetic (with
// run-time flags the arms were all evaluated and selected, tripling the FP64
// work of complex128 rotations).
template <bool SCALED, bool ODD, typename T, typename R>
__device__ __forceinline__ T pauli_upd(T a, T b, R c, R u) {
    T r;
    if (SCALED) {
        if (ODD) {
            r.x = fma_r(-u, b.y, a.x);
            r.y = fma_r(u, b.x, a.y);
        } else {
            r.x = fma_r(u, b.x, a.x);
            r.y = fma_r(u, b.y, a.y);
        }
    } else if (ODD) {
        r.x = c * a.x - u * b.y;
        r.y = c * a.y + u * b.x;
    } else {
        r.x = c * a.x + u * b.x;
        r.y = c * a.y + u * b.y;
    }
    return r;
}

template <bool SCALED, bool ODD, typename T, int NT, typename R>
__device__ __forceinline__ void pauli_pass(T *tile, int m, unsigned x, unsigned z, R c, R w) {
    const unsigned Nt = 1u << m;
    if (x == 0) {
        for (unsigned j = threadIdx.x; j < Nt; j += NT) {
            const R u = flip_sign(w, __popc(j & z) & 1u);
            const T a = tile[j];
            tile[j] = pauli_upd<SCALED, ODD>(a, a, c, u);
        }
        return;
    }
    const int low = __ffs(x) - 1;
    // U pairs per thread per iteration, all loaded before any is stored (the
    // pairs are disjoint), so shared-memory latency overlaps across them
    constexpr int U = 4;
    const unsigned P = Nt / 2;
    for (unsigned g0 = threadIdx.x; g0 < P; g0 += U * NT) {
        unsigned jj[U];
        T aj[U], ak[U];
#pragma unroll
        for (int u = 0; u < U; u++) {
            const unsigned g = g0 + u * NT;
            jj[u] = ins0(g < P ? g : 0, low);
            aj[u] = tile[jj[u]];
            ak[u] = tile[jj[u] ^ x];
        }
#pragma unroll
        for (int u = 0; u < U; u++) {
            if (g0 + u * NT >= P) break;
            const unsigned j = jj[u], k = j ^ x;
            const R wk = flip_sign(w, __popc(k & z) & 1u);  // W (-1)^{parity(k & z) ^ b}
            const R wj = flip_sign(w, __popc(j & z) & 1u);
            tile[j] = pauli_upd<SCALED, ODD>(aj[u], ak[u], c, wk);
            tile[k] = pauli_upd<SCALED, ODD>(ak[u], aj[u], c, wj);
        }
    }
}

template <typename T, int NT>
__device__ __forceinline__ void apply_pauli(T *tile, int m, const DevOp &op, const T *mats, uint32_t bid) {
    const unsigned x = op.lq[0] | ((unsigned)op.lq[1] << 8);
    const unsigned z = op.lq[2] | ((unsigned)op.lq[3] << 8);
    const bool odd = op.lq[4] & 1;
    const uint32_t zc = op.flags | ((uint32_t)op.pad << 16);
    const bool scaled = op.lq[4] & 2;
    const T cs = mats[op.mat];
    const auto c = cs.x;
    const auto w = flip_sign(cs.y, __popc(zc & bid) & 1u);
    if (scaled) {
        if (odd) pauli_pass<true, true, T, NT>(tile, m, x, z, c, w);
        else pauli_pass<true, false, T, NT>(tile, m, x, z, c, w);
    } else {
        if (odd) pauli_pass<false, true, T, NT>(tile, m, x, z, c, w);
        else pauli_pass<false, false, T, NT>(tile, m, x, z, c, w);
    }
}

// STAGE: matrices come from global memory (k >= 3 ones are staged in mbuf);
// otherwise `mats` is the pass's coefficient slice already in shared memory.
template <typename T, int NT, int KMAX, bool STAGE = true>
__device__ __forceinline__ void apply_op(T *tile, int m, const DevOp &op, const T *mats, T *mbuf,
                                         uint32_t bid) {
    switch (op.k) {
        case 7: apply_pauli<T, NT>(tile, m, op, mats, bid); break;
        case 1: apply_dense_reg<1, T, NT>(tile, m, op, mats); break;
        case 2: apply_dense_reg<2, T, NT>(tile, m, op, mats); break;
        case kMono1: apply_mono<1, T, NT>(tile, m, op, mats); break;
        case kMono2: apply_mono<2, T, NT>(tile, m, op, mats); break;
        case 3: if constexpr (KMAX >= 3) apply_dense_smem<3, T, NT, STAGE>(tile, m, op, mats, mbuf); break;
        case 4: if constexpr (KMAX >= 4) apply_dense_smem<4, T, NT, STAGE>(tile, m, op, mats, mbuf); break;
        case 5: if constexpr (KMAX >= 5) apply_dense_smem<5, T, NT, STAGE>(tile, m, op, mats, mbuf); break;
        default: break;
    }
}

// Programmatic dependent launch: a tile pass is launched while the previous
// kernel on the stream is still running; it stages its program slice first
// and waits for the previous grid (its completion and memory) before it
// touches the state or the control block.  In a kernel launched without the
// attribute the wait returns at once.
__device__ __forceinline__ void grid_dep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void grid_dep_launch_next() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// Asynchronous global -> shared copies (cp.async): issued without waiting,
// completed by cp_async_wait_all (commit + wait for all of this thread's groups).
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async8(void *smem, const void *gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}

__device__ __forceinline__ DevOp load_op(const DevOp *p) {
    uint4 v = __ldg(reinterpret_cast<const uint4 *>(p));
    DevOp o;
    *reinterpret_cast<uint4 *>(&o) = v;
    return o;
}

// ------------------------------------------------------------ tile pass --
// One pass: its op slice ops[0, n_ops) and coefficient slice (mat_count
// complex values starting at element mat_first of the pool; op.mat is relative
// to mat_first) are copied into shared memory together with the tile.

constexpr int kMaxHi = 1024;  // 2^(m - L) entries, m - L <= 10

template <typename R, int NT, int KMAX>
__device__ __forceinline__ void tile_pass_body(const TileArgs &a, const uint64_t bid,
                                               unsigned char *smem_raw) {
    using T = typename V2<R>::T;
    T *tile = reinterpret_cast<T *>(smem_raw);
    T *mats_s = tile + (1u << a.m);                                   // kPassMats values
    DevOp *ops_s = reinterpret_cast<DevOp *>(mats_s + kPassMats);     // kPassOps ops
    __shared__ uint64_t hi_off[kMaxHi];
    grid_dep_launch_next();
    // 1. the pass's ops and coefficients: asynchronous copies
    for (unsigned i = threadIdx.x; i < a.n_ops; i += NT) cp_async16(ops_s + i, a.ops + i);
    {
        const T *gm = reinterpret_cast<const T *>(a.mats) + a.mat_first;
        for (unsigned i = threadIdx.x; i < a.mat_count; i += NT) {
            if constexpr (sizeof(T) == 16) cp_async16(mats_s + i, gm + i);
            else cp_async8(mats_s + i, gm + i);
        }
    }
    // 2. global offsets of the tile rows: the tile origin spreads blockIdx over
    //    the non-pivot positions; tile bits above the L contiguous low ones
    //    (unit basis vectors) add their basis vectors
    uint64_t base = 0;
    for (int j = 0; j < a.n - a.m; j++) base |= ((bid >> j) & 1ull) << a.ntq[j];
    const int L = a.L, hib = a.m - L;
    for (int r = threadIdx.x; r < (1 << hib); r += NT) {
        uint64_t o = base;
        for (int j = 0; j < hib; j++)
            if ((r >> j) & 1) o ^= a.bv[L + j];
        hi_off[r] = o;
    }
    grid_dep_wait();
    const int status = a.ctl->status;  // checked once everything is in flight
    __syncthreads();
    T *st = reinterpret_cast<T *>(a.state);
    const unsigned Nt = 1u << a.m, Lmask = (1u << L) - 1u;
    // 3. gather: 16-byte chunks (two c64 / one c128 amplitude) are contiguous in
    //    global memory whenever the tile holds qubit 0 (L >= 1) or amplitudes
    //    are 16 B; every copy of the tile is in flight at once
    constexpr unsigned per = 16 / sizeof(T);
    const bool vec = sizeof(T) == 16 || L >= 1;
    if (vec) {
        for (unsigned p = threadIdx.x; p < Nt / per; p += NT) {
            const unsigned l = p * per;
            cp_async16(tile + l, st + (hi_off[l >> L] | (l & Lmask)));
        }
    } else {
        for (unsigned l = threadIdx.x; l < Nt; l += NT) cp_async8(tile + l, st + (hi_off[l >> L] | (l & Lmask)));
    }
    cp_async_wait_all();
    __syncthreads();
    if (status) return;  // a failed assertion earlier on this stream: leave the state
    for (uint32_t i = 0; i < a.n_ops; i++) {
        const DevOp op = ops_s[i];
        apply_op<T, NT, KMAX, false>(tile, a.m, op, mats_s, nullptr, (uint32_t)bid);
        __syncthreads();
    }
    if (a.wscale != 1.0) {  // times the cosines of the pass's scaled rotations
        const R sc = (R)a.wscale;
        if (vec) {
            for (unsigned p = threadIdx.x; p < Nt / per; p += NT) {
                const unsigned l = p * per;
                T v[per];
#pragma unroll
                for (unsigned e = 0; e < per; e++) {
                    v[e] = tile[l + e];
                    v[e].x *= sc;
                    v[e].y *= sc;
                }
                *reinterpret_cast<uint4 *>(st + (hi_off[l >> L] | (l & Lmask))) = *reinterpret_cast<const uint4 *>(v);
            }
        } else {
            for (unsigned l = threadIdx.x; l < Nt; l += NT) {
                T v = tile[l];
                v.x *= sc;
                v.y *= sc;
                st[hi_off[l >> L] | (l & Lmask)] = v;
            }
        }
        return;
    }
    if (vec) {
        for (unsigned p = threadIdx.x; p < Nt / per; p += NT) {
            const unsigned l = p * per;
            *reinterpret_cast<uint4 *>(st + (hi_off[l >> L] | (l & Lmask))) =
                *reinterpret_cast<const uint4 *>(tile + l);
        }
    } else {
        for (unsigned l = threadIdx.x; l < Nt; l += NT) st[hi_off[l >> L] | (l & Lmask)] = tile[l];
    }
}

template <typename R, int NT, int KMAX>
__global__ void __launch_bounds__(NT, NT >= 512 || KMAX <= 2 ? 2 : 1) k_tile_pass(TileArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    tile_pass_body<R, NT, KMAX>(a, blockIdx.x, smem_raw);
}

// ------------------------------------------------------ register segments --
// complex64 rotation passes over a tile of 2^m amplitudes (10 <= m <= 14):
// 2^(m-5) threads of 32 amplitudes each.  The pass is a list of segments: a
// kSegMarker op naming 5 tile positions R (the register positions), then
// rotations whose X coordinates lie within R.  In a segment the thread's bits
// run over the other m - 5 tile positions in ascending order (its lanes over
// the lowest of them) and its 32 register slots over R, so a rotation is a
// butterfly between slots s and s ^ xr of one thread: no shared memory and no
// barrier.  The first segment gathers its amplitudes straight from global
// memory and the last scatters them back; shared memory holds the tile only
// to lay it out again between segments.
constexpr int kRegAmps = 32;

__host__ __device__ constexpr int top_bit(int v) { return v >= 16 ? 4 : v >= 8 ? 3 : v >= 4 ? 2 : v >= 2 ? 1 : 0; }

__host__ __device__ constexpr int pair_lo(int p, int H) {  // p with a zero inserted at bit H
    return ((p >> H) << (H + 1)) | (p & ((1 << H) - 1));
}

// Pairs (j, k = j ^ XR), j with XR's top bit clear, coefficient u[p] from the
// rotation's table (see RegRot); in the scaled form (the cosine is applied
// once per pass):
//   ODD:  a'_j = a_j + i u a_k,   a'_k = a_k + i u a_j
//   EVEN: a'_j = a_j - u a_k,     a'_k = a_k + u a_j
template <int XR, bool ODD>
__device__ __forceinline__ void rot_reg(float2 *a, const float4 *U) {
    constexpr int H = top_bit(XR);
    float u[16];
#pragma unroll
    for (int q = 0; q < 4; q++) {
        const float4 v = U[q];
        u[4 * q] = v.x;
        u[4 * q + 1] = v.y;
        u[4 * q + 2] = v.z;
        u[4 * q + 3] = v.w;
    }
#pragma unroll
    for (int p = 0; p < 16; p++) {
        const int j = pair_lo(p, H);
        const int k = j ^ XR;
        const float2 aj = a[j], ak = a[k];
        const float uj = u[p];
        if (ODD) {
            a[j] = make_float2(fmaf(-uj, ak.y, aj.x), fmaf(uj, ak.x, aj.y));
            a[k] = make_float2(fmaf(-uj, aj.y, ak.x), fmaf(uj, aj.x, ak.y));
        } else {
            a[j] = make_float2(fmaf(-uj, ak.x, aj.x), fmaf(-uj, ak.y, aj.y));
            a[k] = make_float2(fmaf(uj, aj.x, ak.x), fmaf(uj, aj.y, ak.y));
        }
    }
}

// No X part: a'_j = (1 + u_j (odd ? i : 1)) a_j, u_j from the 32-entry table.
__device__ __forceinline__ void rot_reg_diag(float2 *a, const float4 *U, bool odd) {
#pragma unroll
    for (int q = 0; q < 8; q++) {
        const float4 v = U[q];
        const float u[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int e = 0; e < 4; e++) {
            const int j = 4 * q + e;
            const float2 w = a[j];
            if (odd) a[j] = make_float2(fmaf(-u[e], w.y, w.x), fmaf(u[e], w.x, w.y));
            else a[j] = make_float2(fmaf(u[e], w.x, w.x), fmaf(u[e], w.y, w.y));
        }
    }
}

// sel = xr << 1 | odd (of a RegRot), xr != 0.
__device__ __forceinline__ void rot_reg_dispatch(float2 *a, unsigned sel, const float4 *U) {
    switch (sel) {
#define QSIM_R(v)                                    \
    case 2 * v: rot_reg<v, false>(a, U); break;      \
    case 2 * v + 1: rot_reg<v, true>(a, U); break;
        QSIM_R(1) QSIM_R(2) QSIM_R(3) QSIM_R(4) QSIM_R(5) QSIM_R(6) QSIM_R(7) QSIM_R(8)
        QSIM_R(9) QSIM_R(10) QSIM_R(11) QSIM_R(12) QSIM_R(13) QSIM_R(14) QSIM_R(15)
        QSIM_R(16) QSIM_R(17) QSIM_R(18) QSIM_R(19) QSIM_R(20) QSIM_R(21) QSIM_R(22)
        QSIM_R(23) QSIM_R(24) QSIM_R(25) QSIM_R(26) QSIM_R(27) QSIM_R(28) QSIM_R(29)
        QSIM_R(30) QSIM_R(31)
#undef QSIM_R
        default: break;
    }
}

// ---- dense 1- and 2-qubit ops on register slots (RegDense) --
// C1 on slot S: pairs (j, j | 2^S); each output summed with cmac from zero in
// column order, as the shared-memory kernel does.
template <int S>
__device__ __forceinline__ void c1_reg(float2 *a, const float2 *M) {
    const float4 r0 = *reinterpret_cast<const float4 *>(M), r1 = *reinterpret_cast<const float4 *>(M + 2);
    const float2 m00 = make_float2(r0.x, r0.y), m01 = make_float2(r0.z, r0.w);
    const float2 m10 = make_float2(r1.x, r1.y), m11 = make_float2(r1.z, r1.w);
#pragma unroll
    for (int p = 0; p < 16; p++) {
        const int j = pair_lo(p, S), k = j | (1 << S);
        const float2 x0 = a[j], x1 = a[k];
        float2 y0 = make_float2(0.f, 0.f), y1 = y0;
        cmac(y0, m00, x0);
        cmac(y0, m01, x1);
        cmac(y1, m10, x0);
        cmac(y1, m11, x1);
        a[j] = y0;
        a[k] = y1;
    }
}

// C2 on slots S0 < S1 (bit 0 of the local index <-> S0): 8 groups of 4.
template <int S0, int S1>
__device__ __forceinline__ void c2_reg(float2 *a, const float2 *M) {
    float2 m[16];
#pragma unroll
    for (int i = 0; i < 8; i++) {
        const float4 v = reinterpret_cast<const float4 *>(M)[i];
        m[2 * i] = make_float2(v.x, v.y);
        m[2 * i + 1] = make_float2(v.z, v.w);
    }
#pragma unroll
    for (int g = 0; g < 8; g++) {
        const int b = pair_lo(pair_lo(g, S0), S1);
        const int idx[4] = {b, b | (1 << S0), b | (1 << S1), b | (1 << S0) | (1 << S1)};
        float2 x[4];
#pragma unroll
        for (int c = 0; c < 4; c++) x[c] = a[idx[c]];
#pragma unroll
        for (int r = 0; r < 4; r++) {
            float2 acc = make_float2(0.f, 0.f);
#pragma unroll
            for (int c = 0; c < 4; c++) cmac(acc, m[4 * r + c], x[c]);
            a[idx[r]] = acc;
        }
    }
}

// Monomial C1 on slot S: out_r = M[r][perm_r] x_{perm_r}.
template <int S>
__device__ __forceinline__ void mono1_reg(float2 *a, const float2 *M, unsigned perm) {
    const unsigned c0 = perm & 1u, c1 = (perm >> 2) & 1u;
    const float2 m0 = M[c0], m1 = M[2 + c1];
#pragma unroll
    for (int p = 0; p < 16; p++) {
        const int j = pair_lo(p, S), k = j | (1 << S);
        const float2 x0 = a[j], x1 = a[k];
        float2 y0 = make_float2(0.f, 0.f), y1 = y0;
        cmac(y0, m0, c0 ? x1 : x0);
        cmac(y1, m1, c1 ? x1 : x0);
        a[j] = y0;
        a[k] = y1;
    }
}

// Monomial C2 on slots S0 < S1 whose nonzero entries follow one of three
// column patterns P, chosen at compile time (no runtime selects):
//   P = 0  diagonal, columns (0, 1, 2, 3);
//   P = 1  rows 1 and 3 exchange columns, (0, 3, 2, 1): a CX controlled by
//          the lower slot, times a diagonal;
//   P = 2  rows 2 and 3 exchange columns, (0, 1, 3, 2): controlled by the
//          higher slot.
// out_r = M[r][col_r] x_{col_r}.  Other monomials run as dense C2s.
__host__ __device__ constexpr int mono_col(int P, int r) {
    return P == 1 ? (r == 1 ? 3 : r == 3 ? 1 : r) : P == 2 ? (r == 2 ? 3 : r == 3 ? 2 : r) : r;
}
template <int S0, int S1, int P>
__device__ __forceinline__ void mono2_reg(float2 *a, const float2 *M) {
    float2 m[4];
#pragma unroll
    for (int r = 0; r < 4; r++) m[r] = M[4 * r + mono_col(P, r)];
#pragma unroll
    for (int g = 0; g < 8; g++) {
        const int b = pair_lo(pair_lo(g, S0), S1);
        const int idx[4] = {b, b | (1 << S0), b | (1 << S1), b | (1 << S0) | (1 << S1)};
        float2 x[4];
#pragma unroll
        for (int c = 0; c < 4; c++) x[c] = a[idx[c]];
#pragma unroll
        for (int r = 0; r < 4; r++) {
            float2 acc = make_float2(0.f, 0.f);
            cmac(acc, m[r], x[mono_col(P, r)]);
            a[idx[r]] = acc;
        }
    }
}

__device__ __forceinline__ void dense_reg_dispatch(float2 *a, unsigned sel, unsigned perm, const float2 *M) {
    switch (sel) {
        case 0: c1_reg<0>(a, M); break;
        case 1: c1_reg<1>(a, M); break;
        case 2: c1_reg<2>(a, M); break;
        case 3: c1_reg<3>(a, M); break;
        case 4: c1_reg<4>(a, M); break;
        case 5: c2_reg<0, 1>(a, M); break;
        case 6: c2_reg<0, 2>(a, M); break;
        case 7: c2_reg<0, 3>(a, M); break;
        case 8: c2_reg<0, 4>(a, M); break;
        case 9: c2_reg<1, 2>(a, M); break;
        case 10: c2_reg<1, 3>(a, M); break;
        case 11: c2_reg<1, 4>(a, M); break;
        case 12: c2_reg<2, 3>(a, M); break;
        case 13: c2_reg<2, 4>(a, M); break;
        case 14: c2_reg<3, 4>(a, M); break;
        case 15: mono1_reg<0>(a, M, perm); break;
        case 16: mono1_reg<1>(a, M, perm); break;
        case 17: mono1_reg<2>(a, M, perm); break;
        case 18: mono1_reg<3>(a, M, perm); break;
        case 19: mono1_reg<4>(a, M, perm); break;
        case 20: mono2_reg<0, 1, 0>(a, M); break;
        case 21: mono2_reg<0, 2, 0>(a, M); break;
        case 22: mono2_reg<0, 3, 0>(a, M); break;
        case 23: mono2_reg<0, 4, 0>(a, M); break;
        case 24: mono2_reg<1, 2, 0>(a, M); break;
        case 25: mono2_reg<1, 3, 0>(a, M); break;
        case 26: mono2_reg<1, 4, 0>(a, M); break;
        case 27: mono2_reg<2, 3, 0>(a, M); break;
        case 28: mono2_reg<2, 4, 0>(a, M); break;
        case 29: mono2_reg<3, 4, 0>(a, M); break;
        case 30: mono2_reg<0, 1, 1>(a, M); break;
        case 31: mono2_reg<0, 2, 1>(a, M); break;
        case 32: mono2_reg<0, 3, 1>(a, M); break;
        case 33: mono2_reg<0, 4, 1>(a, M); break;
        case 34: mono2_reg<1, 2, 1>(a, M); break;
        case 35: mono2_reg<1, 3, 1>(a, M); break;
        case 36: mono2_reg<1, 4, 1>(a, M); break;
        case 37: mono2_reg<2, 3, 1>(a, M); break;
        case 38: mono2_reg<2, 4, 1>(a, M); break;
        case 39: mono2_reg<3, 4, 1>(a, M); break;
        case 40: mono2_reg<0, 1, 2>(a, M); break;
        case 41: mono2_reg<0, 2, 2>(a, M); break;
        case 42: mono2_reg<0, 3, 2>(a, M); break;
        case 43: mono2_reg<0, 4, 2>(a, M); break;
        case 44: mono2_reg<1, 2, 2>(a, M); break;
        case 45: mono2_reg<1, 3, 2>(a, M); break;
        case 46: mono2_reg<1, 4, 2>(a, M); break;
        case 47: mono2_reg<2, 3, 2>(a, M); break;
        case 48: mono2_reg<2, 4, 2>(a, M); break;
        case 49: mono2_reg<3, 4, 2>(a, M); break;
        default: break;
    }
}

// The ops of one segment, on this thread's registers: each rotation takes the
// half of its coefficient table that matches the thread's Z parity (RegRot);
// with DENSE, a RegDense op applies its matrix to its slots.
template <bool DENSE>
__device__ __forceinline__ void seg_rotations(float2 *reg, const RegRot *ops, uint32_t count, uint32_t tb,
                                              uint32_t bid, const float *coef) {
    for (uint32_t k = 0; k < count; k++) {
        const RegRot op = ops[k];
        if (DENSE && op.k == kDenseReg) {
            const RegDense d = *reinterpret_cast<const RegDense *>(ops + k);
            dense_reg_dispatch(reg, d.sel, d.perm, reinterpret_cast<const float2 *>(coef + d.tab));
            continue;
        }
        const uint32_t pt = (__popc(tb & op.zt) ^ __popc(op.zc & bid)) & 1u;
        if (op.sel >> 1) {
            rot_reg_dispatch(reg, op.sel, reinterpret_cast<const float4 *>(coef + op.tab + 16 * pt));
        } else {
            rot_reg_diag(reg, reinterpret_cast<const float4 *>(coef + op.tab + 32 * pt), op.sel & 1u);
        }
    }
}

// Slot s of a segment sits at tile index tb | sum of 2^pos[j] over the set
// bits j of s.  The 32 slots are visited in Gray-code order, so each address
// (shared-memory byte offset, or amplitude index by XOR of basis vectors)
// follows from the previous one with one add or XOR.
__host__ __device__ constexpr int gray(int i) { return i ^ (i >> 1); }
__host__ __device__ constexpr int gray_flip(int i) {  // bit that changes from gray(i-1) to gray(i)
    return (i & 1) ? 0 : (i & 2) ? 1 : (i & 4) ? 2 : (i & 8) ? 3 : 4;
}

__device__ __forceinline__ void seg_store_smem(const float2 *reg, uint32_t addr, const uint32_t *d) {
#pragma unroll
    for (int i = 0; i < kRegAmps; i++) {
        if (i) addr = (gray(i) >> gray_flip(i)) & 1 ? addr + d[gray_flip(i)] : addr - d[gray_flip(i)];
        asm volatile("st.shared.v2.f32 [%0], {%1, %2};" ::"r"(addr), "f"(reg[gray(i)].x), "f"(reg[gray(i)].y)
                     : "memory");
    }
}
__device__ __forceinline__ void seg_load_smem(float2 *reg, uint32_t addr, const uint32_t *d) {
#pragma unroll
    for (int i = 0; i < kRegAmps; i++) {
        if (i) addr = (gray(i) >> gray_flip(i)) & 1 ? addr + d[gray_flip(i)] : addr - d[gray_flip(i)];
        asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];" : "=f"(reg[gray(i)].x), "=f"(reg[gray(i)].y) : "r"(addr)
                     : "memory");
    }
}

// One register-segment pass over tile `bid` of the pass described by `a`, run by
// blockDim.x = 2^(m-5) threads.
template <bool DENSE>
__device__ __forceinline__ void rot_pass_body(const TileArgs &a, const uint32_t bid, unsigned char *smem_raw,
                                              uint32_t *bv_s) {
    float2 *tile = reinterpret_cast<float2 *>(smem_raw);
    float2 *mats_s = tile + (1u << a.m);
    DevOp *ops_s = reinterpret_cast<DevOp *>(mats_s + kPassMats);
    grid_dep_launch_next();
    const unsigned tid = threadIdx.x, nt = blockDim.x;  // 2^(m-5) threads
    for (unsigned i = tid; i < a.n_ops; i += nt) cp_async16(ops_s + i, a.ops + i);
    {
        const float2 *gm = reinterpret_cast<const float2 *>(a.mats) + a.mat_first;
        for (unsigned i = tid; i < a.mat_count; i += nt) cp_async8(mats_s + i, gm + i);
    }
    if (tid < 16) bv_s[tid] = (uint32_t)a.bv[tid];  // n <= 32: amplitude indices fit 32 bits
    uint32_t x0 = 0;  // the tile's origin: the tile number spread over the non-pivot positions
    for (int j = 0; j < a.n - a.m; j++) x0 |= ((bid >> j) & 1u) << a.ntq[j];
    cp_async_wait_all();
    grid_dep_wait();
    if (a.ctl->status) return;  // a failed assertion earlier on this stream: leave the state
    __syncthreads();
    float2 *st = reinterpret_cast<float2 *>(a.state);
    const uint32_t tile_sa = (uint32_t)__cvta_generic_to_shared(tile);
    float2 reg[kRegAmps];
    uint32_t sa_prev = 0, sd_prev[5] = {0, 0, 0, 0, 0};
    for (uint32_t i = 0; i < a.n_ops;) {
        const DevOp mk = ops_s[i];  // kSegMarker: lq[0..4] register positions (ascending), flags = #rotations
        const uint32_t nseg = mk.flags;
        const bool first = i == 0;
        const bool last = i + 1 + nseg >= a.n_ops;
        // this thread's tile index: its bits spread over the non-register positions
        uint32_t tb = tid;
#pragma unroll
        for (int j = 0; j < 5; j++) tb = ins0(tb, mk.lq[j]);
        uint32_t sd[5];
#pragma unroll
        for (int j = 0; j < 5; j++) sd[j] = 8u << mk.lq[j];
        const uint32_t sa = tile_sa + 8u * tb;
        if (!first) seg_store_smem(reg, sa_prev, sd_prev);  // the previous segment's layout
        if (!first) __syncthreads();
        if (first || last) {
            uint32_t gd[5];
#pragma unroll
            for (int j = 0; j < 5; j++) gd[j] = bv_s[mk.lq[j]];
            uint32_t gb = x0;
            for (int b = 0; b < a.m; b++)
                if ((tb >> b) & 1u) gb ^= bv_s[b];
            if (first) {
#pragma unroll
                for (int k = 0; k < kRegAmps; k++) {
                    if (k) gb ^= gd[gray_flip(k)];
                    reg[gray(k)] = st[gb];
                }
            } else {
                seg_load_smem(reg, sa, sd);
            }
            seg_rotations<DENSE>(reg, reinterpret_cast<const RegRot *>(ops_s) + i + 1, nseg, tb, bid,
                          reinterpret_cast<const float *>(mats_s));
            if (last) {
                uint32_t g = x0;
                for (int b = 0; b < a.m; b++)
                    if ((tb >> b) & 1u) g ^= bv_s[b];
                const float sc = a.scale;
#pragma unroll
                for (int k = 0; k < kRegAmps; k++) {
                    if (k) g ^= gd[gray_flip(k)];
                    st[g] = make_float2(sc * reg[gray(k)].x, sc * reg[gray(k)].y);
                }
            }
        } else {
            seg_load_smem(reg, sa, sd);
            __syncthreads();  // all reads of this layout before the next one is written
            seg_rotations<DENSE>(reg, reinterpret_cast<const RegRot *>(ops_s) + i + 1, nseg, tb, bid,
                          reinterpret_cast<const float *>(mats_s));
        }
        sa_prev = sa;
#pragma unroll
        for (int j = 0; j < 5; j++) sd_prev[j] = sd[j];
        i += 1 + nseg;
    }
}

template <int NT, int MINB, bool DENSE>
__global__ void __launch_bounds__(NT, MINB) k_rot_pass(TileArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ uint32_t bv_s[16];
    rot_pass_body<DENSE>(a, blockIdx.x, smem_raw, bv_s);
}

// Register-segment passes of several independent states in one launch (all
// with the same tile size m: blockDim.x = 2^(m-5)): descs[j] covers blocks
// [cta_first_j, cta_first_{j+1}); each block finds its state's pass by binary
// search and runs it on tile (blockIdx.x - cta_first_j).
template <int NT, int MINB, bool DENSE>
__global__ void __launch_bounds__(NT, MINB) k_rot_pass_multi(const TileArgs *descs, int n_desc) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ uint32_t bv_s[16];
    __shared__ TileArgs d;
    if (threadIdx.x == 0) {
        int lo = 0, hi = n_desc - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (descs[mid].cta_first <= blockIdx.x) lo = mid;
            else hi = mid - 1;
        }
        d = descs[lo];
    }
    __syncthreads();
    rot_pass_body<DENSE>(d, blockIdx.x - d.cta_first, smem_raw, bv_s);
}

// --------------------------------------------------- final-state shots --
// Shots of the Born distribution without collapse: FP64 partial sums of
// |a_i|^2 over chunks of consecutive indices, their exclusive prefix sums,
// then one warp per shot: shot s draws v from the Philox block at counter
// (s, 1, 0, 0), finds the chunk whose prefix interval holds v * total (binary
// search) and the first index of the chunk whose running sum exceeds it (warp
// scan), and writes the bits of the mask packed in ascending order.
template <typename R>
__global__ void __launch_bounds__(256) k_sample_partials(const void *state, uint32_t chunk, double *partials) {
    using T = typename V2<R>::T;
    const T *a = reinterpret_cast<const T *>(state) + (uint64_t)blockIdx.x * chunk;
    double acc = 0;
    for (uint32_t i = threadIdx.x; i < chunk; i += 256) acc += norm2(a[i]);
    __shared__ double red[256 / 32];
#pragma unroll
    for (int o = 16; o; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0;
        for (int w = 0; w < 256 / 32; w++) t += red[w];
        partials[blockIdx.x] = t;
    }
}

// One block of 1024 threads: offsets[b] = sum of partials[0..b), offsets[P] = total.
__global__ void __launch_bounds__(1024) k_sample_scan(const double *partials, uint32_t P, double *offsets) {
    __shared__ double seg[1024];
    const uint32_t per = (P + 1023) / 1024;
    const uint32_t lo = min(P, threadIdx.x * per), hi = min(P, lo + per);
    double t = 0;
    for (uint32_t i = lo; i < hi; i++) t += partials[i];
    seg[threadIdx.x] = t;
    __syncthreads();
    if (threadIdx.x == 0) {  // exclusive prefix of the 1024 segment sums
        double run = 0;
        for (int i = 0; i < 1024; i++) {
            const double v = seg[i];
            seg[i] = run;
            run += v;
        }
        offsets[P] = run;
    }
    __syncthreads();
    double run = seg[threadIdx.x];
    for (uint32_t i = lo; i < hi; i++) {
        offsets[i] = run;
        run += partials[i];
    }
}

__device__ __forceinline__ uint64_t pack_bits(uint64_t x, uint64_t mask) {
    uint64_t r = 0;
    int j = 0;
    for (int b = 0; b < 64; b++)
        if ((mask >> b) & 1ull) r |= ((x >> b) & 1ull) << j++;
    return r;
}

template <typename R>
__global__ void __launch_bounds__(256) k_sample_draw(const void *state, uint32_t chunk, uint32_t P,
                                                     const double *offsets, uint64_t seed, uint64_t shots,
                                                     uint64_t mask, uint64_t *out) {
    using T = typename V2<R>::T;
    const T *a = reinterpret_cast<const T *>(state);
    const unsigned lane = threadIdx.x & 31;
    const uint64_t warps = (uint64_t)gridDim.x * (blockDim.x >> 5);
    const double total = offsets[P];
    for (uint64_t s = (uint64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); s < shots; s += warps) {
        const double v = (double)(philox_word0(s, seed, 1) >> 11) * (1.0 / 9007199254740992.0);
        const double target = v * total;
        // last chunk whose prefix is <= target
        uint32_t lo = 0, hi = P - 1;
        while (lo < hi) {
            const uint32_t mid = lo + (hi - lo + 1) / 2;
            if (offsets[mid] <= target) lo = mid;
            else hi = mid - 1;
        }
        uint64_t x = ~0ull, last_nz = ~0ull;
        for (uint32_t b = lo; b < P && x == ~0ull; b++) {
            double base = offsets[b];
            const uint64_t first = (uint64_t)b * chunk;
            for (uint32_t j = 0; j < chunk && x == ~0ull; j += 32) {
                const uint32_t i = j + lane;
                const double w = i < chunk ? norm2(a[first + i]) : 0.0;
                double inc = w;  // inclusive warp scan in lane order
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const double t = __shfl_up_sync(0xffffffffu, inc, o);
                    if (lane >= (unsigned)o) inc += t;
                }
                const unsigned hit = __ballot_sync(0xffffffffu, i < chunk && w > 0 && base + inc > target);
                const unsigned nz = __ballot_sync(0xffffffffu, i < chunk && w > 0);
                if (hit) x = first + j + (__ffs(hit) - 1);
                else if (nz) last_nz = first + j + (31 - __clz(nz));
                base += __shfl_sync(0xffffffffu, inc, 31);
            }
        }
        if (x == ~0ull) x = last_nz;  // rounding put the target past the last nonzero entry
        if (lane == 0) out[s] = pack_bits(x == ~0ull ? 0 : x, mask);
    }
}

// ------------------------------------------------ persistent rotation pass --
// The same register-segment pass, run by blocks that stay resident and take
// tiles from a device counter: tile k + 1 of a block is copied into shared
// memory (cp.async, whole 128-byte rows) while tile k is computed in
// registers, so the L2 traffic of one tile overlaps the arithmetic of the
// previous one, and blocks on lightly loaded SMs take more tiles.  Tiles are
// numbered base, base + 1, ... on the counter: a block stops at the first
// number past the pass's last tile, so each launch advances the counter by
// exactly n_tiles + gridDim.x.  Needs the 4 forced low qubits (whole rows).
constexpr int kMaxRows = 1024;  // 2^(m-4) rows, m <= 14

template <int NT>
__global__ void __launch_bounds__(NT, NT <= 64 ? 8 : NT <= 128 ? 4 : 2)
    k_rot_pipe(TileArgs a, unsigned long long *ctr, unsigned long long base, uint32_t n_tiles) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const unsigned Nt = 1u << a.m;
    float2 *bufs = reinterpret_cast<float2 *>(smem_raw);  // two tiles, then the program slices
    float2 *mats_s = bufs + 2 * Nt;
    DevOp *ops_s = reinterpret_cast<DevOp *>(mats_s + ((a.mat_count + 1) & ~1u));
    __shared__ uint32_t bv_s[16];
    __shared__ uint32_t rowL[kMaxRows];   // XOR of the basis vectors of a row's local bits 4..m-1
    __shared__ uint32_t next_tile[2];
    grid_dep_launch_next();
    const unsigned tid = threadIdx.x, nt = blockDim.x;
    for (unsigned i = tid; i < a.n_ops; i += nt) cp_async16(ops_s + i, a.ops + i);
    {
        const float2 *gm = reinterpret_cast<const float2 *>(a.mats) + a.mat_first;
        for (unsigned i = tid; i < a.mat_count; i += nt) cp_async8(mats_s + i, gm + i);
    }
    if (tid < 16) bv_s[tid] = (uint32_t)a.bv[tid];
    const unsigned rows = Nt >> 4;
    for (unsigned r = tid; r < rows; r += nt) {
        uint32_t v = 0;
        for (int j = 0; j < a.m - 4; j++)
            if ((r >> j) & 1u) v ^= (uint32_t)a.bv[4 + j];
        rowL[r] = v;
    }
    cp_async_wait_all();
    grid_dep_wait();
    if (a.ctl->status) {  // a failed assertion earlier on this stream: leave the state, keep the count
        if (tid == 0)
            while (atomicAdd(ctr, 1ull) - base < n_tiles) {
            }
        return;
    }
    if (tid == 0) {
        next_tile[0] = (uint32_t)min(atomicAdd(ctr, 1ull) - base, (unsigned long long)n_tiles);
        next_tile[1] = next_tile[0] < n_tiles ? (uint32_t)min(atomicAdd(ctr, 1ull) - base, (unsigned long long)n_tiles)
                                              : n_tiles;
    }
    __syncthreads();
    float2 *st = reinterpret_cast<float2 *>(a.state);
    // the tile's origin: its number spread over the non-pivot positions
    auto origin = [&](uint32_t t) {
        uint32_t x0 = 0;
        for (int j = 0; j < a.n - a.m; j++) x0 |= ((t >> j) & 1u) << a.ntq[j];
        return x0;
    };
    // copy tile t into buf as whole rows in address order
    auto prefetch = [&](uint32_t t, float2 *buf) {
        const uint32_t x0 = origin(t);
        for (unsigned c = tid; c < Nt / 2; c += nt) {  // 16-byte chunks, 8 per row
            const unsigned r = c >> 3;
            const uint32_t row = (x0 ^ rowL[r]) & ~15u;
            cp_async16(buf + 2 * c, st + row + 2 * (c & 7));
        }
        asm volatile("cp.async.commit_group;\n" ::: "memory");
    };
    uint32_t cur = next_tile[0];
    if (cur < n_tiles) prefetch(cur, bufs);
    float2 reg[kRegAmps];
    for (uint32_t k = 0; cur < n_tiles; k++) {
        float2 *buf = bufs + (k & 1) * Nt;
        asm volatile("cp.async.wait_group 0;\n" ::: "memory");
        __syncthreads();  // tile k in place; the other buffer's last readers are done
        const uint32_t nxt = next_tile[(k + 1) & 1];
        if (tid == 0 && nxt < n_tiles)
            next_tile[k & 1] = (uint32_t)min(atomicAdd(ctr, 1ull) - base, (unsigned long long)n_tiles);
        if (nxt < n_tiles) prefetch(nxt, bufs + ((k + 1) & 1) * Nt);
        const uint32_t bid = cur;
        const uint32_t x0 = origin(cur);
        const uint32_t tile_sa = (uint32_t)__cvta_generic_to_shared(buf);
        uint32_t sa_prev = 0, sd_prev[5] = {0, 0, 0, 0, 0};
        for (uint32_t i = 0; i < a.n_ops;) {
            const DevOp mk = ops_s[i];
            const uint32_t nseg = mk.flags;
            const bool first = i == 0;
            const bool last = i + 1 + nseg >= a.n_ops;
            uint32_t tb = tid;
#pragma unroll
            for (int j = 0; j < 5; j++) tb = ins0(tb, mk.lq[j]);
            uint32_t sd[5];
#pragma unroll
            for (int j = 0; j < 5; j++) sd[j] = 8u << mk.lq[j];
            const uint32_t sa = tile_sa + 8u * tb;
            if (first) {
                // rows sit in address order: local index l at l ^ (rowL[l >> 4] & 15)
                uint32_t pd[5];
#pragma unroll
                for (int j = 0; j < 5; j++) {
                    const uint32_t u = 1u << mk.lq[j];
                    pd[j] = 8u * (u ^ (u >= 16 ? bv_s[mk.lq[j]] & 15u : 0u));
                }
                uint32_t tphys = tb;
                for (int b = 4; b < a.m; b++)
                    if ((tb >> b) & 1u) tphys ^= bv_s[b] & 15u;
                uint32_t off = 8u * tphys;
#pragma unroll
                for (int q = 0; q < kRegAmps; q++) {
                    if (q) off ^= pd[gray_flip(q)];
                    asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];"
                                 : "=f"(reg[gray(q)].x), "=f"(reg[gray(q)].y)
                                 : "r"(tile_sa + off)
                                 : "memory");
                }
                if (!last) __syncthreads();  // every first-layout read before the tile is re-laid out
            } else {
                seg_store_smem(reg, sa_prev, sd_prev);
                __syncthreads();
                seg_load_smem(reg, sa, sd);
                if (!last) __syncthreads();
            }
            seg_rotations<false>(reg, reinterpret_cast<const RegRot *>(ops_s) + i + 1, nseg, tb, bid,
                          reinterpret_cast<const float *>(mats_s));
            if (last) {
                uint32_t gd[5];
#pragma unroll
                for (int j = 0; j < 5; j++) gd[j] = bv_s[mk.lq[j]];
                uint32_t g = x0;
                for (int b = 0; b < a.m; b++)
                    if ((tb >> b) & 1u) g ^= bv_s[b];
                const float sc = a.scale;
#pragma unroll
                for (int q = 0; q < kRegAmps; q++) {
                    if (q) g ^= gd[gray_flip(q)];
                    st[g] = make_float2(sc * reg[gray(q)].x, sc * reg[gray(q)].y);
                }
            }
            sa_prev = sa;
#pragma unroll
            for (int j = 0; j < 5; j++) sd_prev[j] = sd[j];
            i += 1 + nseg;
        }
        cur = nxt;
    }
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
}

// One pass of several independent states in one launch: descs[j] covers
// blocks [cta_first_j, cta_first_{j+1}); each block finds its state's pass by
// binary search and runs it on tile (blockIdx.x - cta_first_j).
template <typename R, int NT, int KMAX>
__global__ void __launch_bounds__(NT, NT >= 512 || KMAX <= 2 ? 2 : 1) k_tile_pass_multi(const TileArgs *descs,
                                                                            int n_desc) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ TileArgs d;
    if (threadIdx.x == 0) {
        int lo = 0, hi = n_desc - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (descs[mid].cta_first <= blockIdx.x) lo = mid;
            else hi = mid - 1;
        }
        d = descs[lo];
    }
    __syncthreads();
    tile_pass_body<R, NT, KMAX>(d, blockIdx.x - d.cta_first, smem_raw);
}

// -------------------------------------------------------------- resident --
template <typename T, int NT, int KMAX>
__device__ void run_resident(const Instance &in, T *tile, double *red, int *bcast, double *bscale,
                             int max_n) {
    const int n = in.n;
    const unsigned N = 1u << n;
    T *mbuf = tile + (1u << max_n);
    T *st = reinterpret_cast<T *>(in.state);
    if (in.flags & kInstInit) {
        // start from |0...0> with a cleared control block: no state read at all
        for (unsigned l = threadIdx.x; l < N; l += NT) {
            T v = czero(tile[0]);
            if (l == 0) v.x = 1;
            tile[l] = v;
        }
        if (threadIdx.x == 0) {
            in.ctl->status = 0;
            in.ctl->success = 1.0;
            in.ctl->arrive = 0;
        }
    } else {
        if (in.ctl->status) return;
        for (unsigned l = threadIdx.x; l < N; l += NT) tile[l] = st[l];
    }
    __syncthreads();
    const T *mats = reinterpret_cast<const T *>(in.mats);
    uint64_t ev = 0;
    bool failed = false;
    DevOp nxt = load_op(in.ops);
    for (uint64_t i = 0; i < in.n_ops; i++) {
        const DevOp op = nxt;
        if (i + 1 < in.n_ops) nxt = load_op(in.ops + i + 1);  // in flight while op runs
        if (op.k) {
            apply_op<T, NT, KMAX>(tile, n, op, mats, mbuf, 0u);
            __syncthreads();
            continue;
        }
        // measurement / reset on qubit q
        const int q = op.lq[0];
        double s0 = 0, s1 = 0;
        for (unsigned l = threadIdx.x; l < N; l += NT) {
            const double w = norm2_term(tile[l]);
            if ((l >> q) & 1u) s1 += w;
            else s0 += w;
        }
        block_sum2<NT>(s0, s1, red);
        const int reset = op.ev == 2;
        if (threadIdx.x == 0) {
            Decision d = decide(s0, s1, op.flags, reset, in.seed, in.ordinal0 + ev, in.thr);
            const uint64_t li = in.log0 + ev;
            if (li < in.log_cap) {
                in.log[li].outcome = d.outcome;
                in.log[li].prob = d.prob;
            }
            if (d.fail) {
                in.ctl->status = 4;  // QSIM_E_ZEROPROB
                in.ctl->fail_log = li;
            } else if ((op.flags & 1) && !reset) {
                in.ctl->success *= d.prob;
            }
            in.ctl->p0 = s0;
            in.ctl->p1 = s1;
            bcast[0] = d.fail ? -1 : d.outcome;
            bscale[0] = d.scale;
        }
        __syncthreads();
        const int outc = bcast[0];
        const double sc = bscale[0];
        __syncthreads();
        ev++;
        if (outc < 0) {
            failed = true;
            break;
        }
        const unsigned bq = 1u << q;
        for (unsigned i2 = threadIdx.x; i2 < N / 2; i2 += NT) {
            const unsigned i0 = ins0(i2, q), i1 = i0 | bq;
            const T a0 = tile[i0], a1 = tile[i1];
            if (outc == 0) {
                tile[i0] = scale_by(a0, sc);
            } else if (reset) {
                tile[i0] = scale_by(a1, sc);
            } else {
                tile[i0] = czero(a0);
            }
            tile[i1] = (outc == 1 && !reset) ? scale_by(a1, sc) : czero(a1);
        }
        __syncthreads();
    }
    (void)failed;
    for (unsigned l = threadIdx.x; l < N; l += NT) st[l] = tile[l];
}

template <typename R, int NT, int KMAX>
__global__ void __launch_bounds__(NT) k_resident_one(Instance in) {
    using T = typename V2<R>::T;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double red[2 * NT / 32];
    __shared__ int bcast[1];
    __shared__ double bscale[1];
    run_resident<T, NT, KMAX>(in, reinterpret_cast<T *>(smem_raw), red, bcast, bscale, in.n);
}

template <typename R, int NT, int KMAX>
__global__ void __launch_bounds__(NT) k_resident_batch(const Instance *insts, int max_n) {
    using T = typename V2<R>::T;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double red[2 * NT / 32];
    __shared__ int bcast[1];
    __shared__ double bscale[1];
    const Instance in = insts[blockIdx.x];
    run_resident<T, NT, KMAX>(in, reinterpret_cast<T *>(smem_raw), red, bcast, bscale, max_n);
}

// ----------------------------------------------------------- measurement --
constexpr int kRedThreads = 256;

template <typename R, bool DECIDE>
__global__ void __launch_bounds__(kRedThreads) k_prob(const void *state, int n, MeasArgs a,
                                                      double *partials, MeasCtl *ctl, MeasRec *log) {
    using T = typename V2<R>::T;
    __shared__ double red[2 * kRedThreads / 32];
    __shared__ int last;
    if (ctl->status) return;
    const T *st = reinterpret_cast<const T *>(state);
    const uint64_t N = 1ull << n;
    const uint64_t chunk = N / gridDim.x;
    const uint64_t start = chunk * blockIdx.x;
    double s0 = 0, s1 = 0;
    for (uint64_t l = threadIdx.x; l < chunk; l += kRedThreads) {
        const uint64_t i = start + l;
        const double w = norm2_term(st[i]);
        if ((i >> a.q) & 1ull) s1 += w;
        else s0 += w;
    }
    block_sum2<kRedThreads>(s0, s1, red);
    if (threadIdx.x == 0) {
        partials[2 * blockIdx.x] = s0;
        partials[2 * blockIdx.x + 1] = s1;
        __threadfence();
        const unsigned t = atomicAdd(&ctl->arrive, 1u);
        last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    // the block partials in a fixed shape: thread t sums blocks t, t + 256, ...
    // in order, then the warp-shuffle / warp-order tree of block_sum2, so the
    // result depends only on the grid size (no serial chain over all blocks)
    double x = 0, y = 0;
    for (unsigned b = threadIdx.x; b < gridDim.x; b += kRedThreads) {
        x += __ldcg(partials + 2 * b);
        y += __ldcg(partials + 2 * b + 1);
    }
    block_sum2<kRedThreads>(x, y, red);
    if (threadIdx.x == 0) {
        ctl->arrive = 0;
        ctl->p0 = x;
        ctl->p1 = y;
        if (DECIDE) {
            Decision d = decide(x, y, a.mode, a.reset, a.seed, a.ordinal, a.thr);
            if (a.log_idx < a.log_cap) {
                log[a.log_idx].outcome = d.outcome;
                log[a.log_idx].prob = d.prob;
            }
            if (d.fail) {
                ctl->status = 4;  // QSIM_E_ZEROPROB
                ctl->fail_log = a.log_idx;
            } else if ((a.mode & 1) && !a.reset) {
                ctl->success *= d.prob;
            }
            ctl->outcome = d.outcome;
            ctl->scale = d.scale;
        }
    }
}

template <typename R>
__global__ void __launch_bounds__(256) k_collapse(void *state, int n, int q, int reset,
                                                  const MeasCtl *ctl) {
    using T = typename V2<R>::T;
    if (ctl->status) return;
    const int outc = ctl->outcome;
    const double sc = ctl->scale;
    T *st = reinterpret_cast<T *>(state);
    const uint64_t half = 1ull << (n - 1), bq = 1ull << q;
    for (uint64_t i = blockIdx.x * 256ull + threadIdx.x; i < half; i += (uint64_t)gridDim.x * 256ull) {
        const uint64_t i0 = ins0_64(i, q), i1 = i0 | bq;
        const T a0 = st[i0], a1 = st[i1];
        if (outc == 0) st[i0] = scale_by(a0, sc);
        else if (reset) st[i0] = scale_by(a1, sc);
        else st[i0] = czero(a0);
        st[i1] = (outc == 1 && !reset) ? scale_by(a1, sc) : czero(a1);
    }
}

// ----------------------------------------------------------- expectation --
template <typename R>
__global__ void __launch_bounds__(256) k_expect(const void *state, int n, const uint64_t *terms,
                                                double *partials) {
    using T = typename V2<R>::T;
    __shared__ double red[2 * 256 / 32];
    const T *st = reinterpret_cast<const T *>(state);
    const uint64_t x = terms[3 * blockIdx.y], z = terms[3 * blockIdx.y + 1];
    const int ny = __popcll(x & z) & 3;
    const uint64_t N = 1ull << n, chunk = N / gridDim.x, start = chunk * blockIdx.x;
    double acc = 0, dummy = 0;
    for (uint64_t l = threadIdx.x; l < chunk; l += 256) {
        const uint64_t j = start + l;
        // Re(i^ny conj(a_{j^x}) a_j) (-1)^{parity(j & z)}
        acc += pauli_term(st[j], st[j ^ x], ny, __popcll(j & z) & 1u);
    }
    block_sum2<256>(acc, dummy, red);
    if (threadIdx.x == 0) partials[(uint64_t)blockIdx.y * gridDim.x + blockIdx.x] = acc;
}

// Batched expectation: block b evaluates every term of job b over its (small)
// state, each term a fixed-shape FP64 block reduction in index order per thread.
template <typename R>
__global__ void __launch_bounds__(256) k_expect_batch(const ExpectJob *jobs) {
    using T = typename V2<R>::T;
    __shared__ double red[2 * 256 / 32];
    const ExpectJob jb = jobs[blockIdx.x];
    const T *st = reinterpret_cast<const T *>(jb.state);
    const uint64_t N = 1ull << jb.n;
    for (uint32_t t = 0; t < jb.n_terms; t++) {
        const uint64_t x = jb.terms[3 * t], z = jb.terms[3 * t + 1];
        const int ny = __popcll(x & z) & 3;
        double acc = 0, dummy = 0;
        for (uint64_t j = threadIdx.x; j < N; j += 256) {
            acc += pauli_term(st[j], st[j ^ x], ny, __popcll(j & z) & 1u);
        }
        block_sum2<256>(acc, dummy, red);
        if (threadIdx.x == 0) jb.out[t] = __longlong_as_double((long long)jb.terms[3 * t + 2]) * acc;
    }
}

__global__ void k_expect_final(const uint64_t *terms, size_t n_terms, int P, const double *partials,
                               double *out) {
    const size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (t >= n_terms) return;
    double s = 0;
    for (int b = 0; b < P; b++) s += partials[t * P + b];
    out[t] = __longlong_as_double((long long)terms[3 * t + 2]) * s;
}

template <typename R>
__global__ void k_set_basis(void *state, uint64_t N, uint64_t index) {
    using T = typename V2<R>::T;
    T *st = reinterpret_cast<T *>(state);
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < N;
         i += (uint64_t)gridDim.x * blockDim.x) {
        T v = czero(st[0]);
        if (i == index) v.x = 1;
        st[i] = v;
    }
}

template <typename R> constexpr size_t amp_bytes() { return sizeof(typename V2<R>::T); }

}  // namespace

// ------------------------------------------------------------- launchers --
int max_resident_bits(int dtype) { return dtype == 0 ? 14 : 13; }

size_t resident_smem_bytes(int dtype, int n) {
    const size_t es = dtype == 0 ? 8 : 16;
    return (es << n) + es * 32 * 32;  // state + one staged k <= 5 matrix
}

cudaError_t setup_kernels() {
    const int big = 227 * 1024;
    cudaError_t e;
#define QSIM_ATTR(fn)                                                                      \
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, big - 24 * 1024); \
    if (e != cudaSuccess) return e;
    QSIM_ATTR((k_tile_pass<float, 256, 2>));
    QSIM_ATTR((k_tile_pass<double, 256, 2>));
    QSIM_ATTR((k_tile_pass<float, 512, 2>));
    QSIM_ATTR((k_tile_pass<double, 512, 2>));
    QSIM_ATTR((k_tile_pass<float, 256, 5>));
    QSIM_ATTR((k_tile_pass<double, 256, 5>));
    QSIM_ATTR((k_rot_pass<128, 4, false>));
    QSIM_ATTR((k_rot_pass<256, 2, false>));
    QSIM_ATTR((k_rot_pass<512, 1, false>));
    QSIM_ATTR((k_rot_pass<128, 4, true>));
    QSIM_ATTR((k_rot_pass<256, 2, true>));
    QSIM_ATTR((k_rot_pass<512, 1, true>));
    QSIM_ATTR((k_rot_pass_multi<128, 4, false>));
    QSIM_ATTR((k_rot_pass_multi<256, 2, false>));
    QSIM_ATTR((k_rot_pass_multi<512, 1, false>));
    QSIM_ATTR((k_rot_pass_multi<128, 4, true>));
    QSIM_ATTR((k_rot_pass_multi<256, 2, true>));
    QSIM_ATTR((k_rot_pass_multi<512, 1, true>));
    QSIM_ATTR(k_rot_pipe<64>);
    QSIM_ATTR(k_rot_pipe<128>);
    QSIM_ATTR(k_rot_pipe<256>);
    QSIM_ATTR((k_tile_pass_multi<float, 256, 2>));
    QSIM_ATTR((k_tile_pass_multi<double, 256, 2>));
    QSIM_ATTR((k_tile_pass_multi<float, 512, 2>));
    QSIM_ATTR((k_tile_pass_multi<double, 512, 2>));
    QSIM_ATTR((k_tile_pass_multi<float, 256, 5>));
    QSIM_ATTR((k_tile_pass_multi<double, 256, 5>));
    QSIM_ATTR((k_resident_one<float, 256, 2>));
    QSIM_ATTR((k_resident_one<double, 256, 2>));
    QSIM_ATTR((k_resident_batch<float, 256, 2>));
    QSIM_ATTR((k_resident_batch<double, 256, 2>));
    QSIM_ATTR((k_resident_one<float, 256, 5>));
    QSIM_ATTR((k_resident_one<double, 256, 5>));
    QSIM_ATTR((k_resident_batch<float, 256, 5>));
    QSIM_ATTR((k_resident_batch<double, 256, 5>));
#undef QSIM_ATTR
    return cudaSuccess;
}

bool make_tile_args(int dtype, void *state, int n, int m, uint64_t pivots, const uint64_t *basis,
                    const DevOp *ops, uint32_t n_ops, const void *mats, uint32_t mat_first,
                    uint32_t mat_count, const MeasCtl *ctl, TileArgs *out) {
    if (n_ops > (uint32_t)kPassOps || mat_count > (uint32_t)kPassMats || m > 15 || n - m > 48 ||
        m < 1 || m > n || n > 63)
        return false;
    TileArgs &a = *out;
    std::memset(&a, 0, sizeof(a));
    a.state = state;
    a.ops = ops;
    a.mats = mats;
    a.ctl = ctl;
    a.n_ops = n_ops;
    a.mat_first = mat_first;
    a.mat_count = mat_count;
    a.n = n;
    a.m = m;
    const uint64_t all = (1ull << n) - 1;
    if (__builtin_popcountll(pivots & all) != m || (pivots & ~all)) return false;
    for (int j = 0; j < m; j++) {
        if (!basis[j] || (basis[j] & ~all)) return false;
        a.bv[j] = basis[j];
    }
    int u = 0;
    for (int b = 0; b < n; b++)
        if (!((pivots >> b) & 1ull)) a.ntq[u++] = (uint8_t)b;
    // contiguous low run of the tile (128-byte rows at most): the leading
    // basis vectors are the unit vectors of qubits 0.. and no later basis
    // vector has a bit below them; a pass may lack such a run
    const int cap = dtype == 0 ? 4 : 3;
    int L = 0;
    while (L < cap && L < m && basis[L] == (1ull << L)) L++;
    for (; L > 0; L--) {
        bool ok = true;
        for (int j = L; j < m; j++)
            if (basis[j] & ((1ull << L) - 1)) ok = false;
        if (ok) break;
    }
    a.L = L;
    a.wscale = 1.0;
    return true;
}

// Launch with programmatic stream serialization (see grid_dep_wait).
template <typename Kern>
cudaError_t launch_dependent(Kern kern, unsigned grid, unsigned block, size_t smem, cudaStream_t s,
                             const TileArgs &a) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, a);
}

bool generic_tile_ok(const TileArgs &a) { return (1 << (a.m - a.L)) <= kMaxHi; }

cudaError_t launch_tile_pass(int dtype, int threads, int kmax, void *state, int n, int m,
                             uint64_t pivots, const uint64_t *basis, const DevOp *ops, uint32_t n_ops,
                             const void *mats, uint32_t mat_first, uint32_t mat_count, double wscale,
                             const MeasCtl *ctl, cudaStream_t s) {
    TileArgs a;
    if (!make_tile_args(dtype, state, n, m, pivots, basis, ops, n_ops, mats, mat_first, mat_count, ctl, &a) ||
        !generic_tile_ok(a))
        return cudaErrorInvalidValue;
    a.wscale = wscale;
    const unsigned grid = 1u << (n - m);
    const size_t smem = tile_smem_bytes(dtype, m);
    if (kmax > 2) {
        if (dtype == 0) return launch_dependent(k_tile_pass<float, 256, 5>, grid, 256, smem, s, a);
        return launch_dependent(k_tile_pass<double, 256, 5>, grid, 256, smem, s, a);
    }
    if (dtype == 0) {
        if (threads == 512) return launch_dependent(k_tile_pass<float, 512, 2>, grid, 512, smem, s, a);
        return launch_dependent(k_tile_pass<float, 256, 2>, grid, 256, smem, s, a);
    }
    if (threads == 512) return launch_dependent(k_tile_pass<double, 512, 2>, grid, 512, smem, s, a);
    return launch_dependent(k_tile_pass<double, 256, 2>, grid, 256, smem, s, a);
}

cudaError_t launch_rot_pass(void *state, int n, int m, uint64_t pivots, const uint64_t *basis,
                            const DevOp *ops, uint32_t n_ops, const void *mats, uint32_t mat_first,
                            uint32_t mat_count, float scale, bool dense, const MeasCtl *ctl, cudaStream_t s) {
    if (m < 10 || m > 14 || n > 32) return cudaErrorInvalidValue;
    TileArgs a;
    if (!make_tile_args(0, state, n, m, pivots, basis, ops, n_ops, mats, mat_first, mat_count, ctl, &a))
        return cudaErrorInvalidValue;
    a.scale = scale;
    const unsigned grid = 1u << (n - m), threads = 1u << (m - 5);
    const size_t smem = tile_smem_bytes(0, m);
    if (dense) {
        if (m == 12) return launch_dependent(k_rot_pass<128, 4, true>, grid, threads, smem, s, a);
        if (m <= 13) return launch_dependent(k_rot_pass<256, 2, true>, grid, threads, smem, s, a);
        return launch_dependent(k_rot_pass<512, 1, true>, grid, threads, smem, s, a);
    }
    if (m == 12) return launch_dependent(k_rot_pass<128, 4, false>, grid, threads, smem, s, a);
    if (m <= 13) return launch_dependent(k_rot_pass<256, 2, false>, grid, threads, smem, s, a);
    return launch_dependent(k_rot_pass<512, 1, false>, grid, threads, smem, s, a);
}

cudaError_t launch_rot_pass_multi(const TileArgs *d_descs, int n_desc, uint32_t total_ctas, int m, bool dense,
                                  cudaStream_t s) {
    if (n_desc <= 0 || total_ctas == 0) return cudaSuccess;
    if (m < 10 || m > 14) return cudaErrorInvalidValue;
    const unsigned threads = 1u << (m - 5);
    const size_t smem = tile_smem_bytes(0, m);
    if (dense) {
        if (m == 12) k_rot_pass_multi<128, 4, true><<<total_ctas, threads, smem, s>>>(d_descs, n_desc);
        else if (m <= 13) k_rot_pass_multi<256, 2, true><<<total_ctas, threads, smem, s>>>(d_descs, n_desc);
        else k_rot_pass_multi<512, 1, true><<<total_ctas, threads, smem, s>>>(d_descs, n_desc);
    } else {
        if (m == 12) k_rot_pass_multi<128, 4, false><<<total_ctas, threads, smem, s>>>(d_descs, n_desc);
        else if (m <= 13) k_rot_pass_multi<256, 2, false><<<total_ctas, threads, smem, s>>>(d_descs, n_desc);
        else k_rot_pass_multi<512, 1, false><<<total_ctas, threads, smem, s>>>(d_descs, n_desc);
    }
    return cudaGetLastError();
}

cudaError_t launch_rot_pipe(void *state, int n, int m, uint64_t pivots, const uint64_t *basis,
                            const DevOp *ops, uint32_t n_ops, const void *mats, uint32_t mat_first,
                            uint32_t mat_count, float scale, const MeasCtl *ctl, unsigned long long *ctr,
                            unsigned long long base, uint32_t *grid_used, cudaStream_t s) {
    if (m < 10 || m > 13 || n > 32) return cudaErrorInvalidValue;
    TileArgs a;
    if (!make_tile_args(0, state, n, m, pivots, basis, ops, n_ops, mats, mat_first, mat_count, ctl, &a))
        return cudaErrorInvalidValue;
    for (int j = 0; j < 4; j++)  // whole 128-byte rows
        if (basis[j] != (1ull << j)) return cudaErrorInvalidValue;
    a.scale = scale;
    const size_t smem = ((size_t)16 << m) + 8 * (size_t)((mat_count + 1) & ~1u) + sizeof(DevOp) * n_ops;
    // resident blocks per SM: shared memory (this launch's plus the static
    // 4.1 KB) and registers (128 per thread)
    const unsigned threads = 1u << (m - 5);
    int per_sm = (int)((227u * 1024u) / (smem + 4352));
    per_sm = std::min(per_sm, (int)(512u / threads));
    per_sm = std::max(per_sm, 1);
    const uint32_t n_tiles = 1u << (n - m);
    const uint32_t grid = std::min<uint32_t>(n_tiles, 152u * (uint32_t)per_sm);
    *grid_used = grid;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(threads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    if (m <= 11) return cudaLaunchKernelEx(&cfg, k_rot_pipe<64>, a, ctr, base, n_tiles);
    if (m == 12) return cudaLaunchKernelEx(&cfg, k_rot_pipe<128>, a, ctr, base, n_tiles);
    return cudaLaunchKernelEx(&cfg, k_rot_pipe<256>, a, ctr, base, n_tiles);
}

int sample_chunk(int n) { return n >= 9 ? 512 : 1 << n; }

cudaError_t launch_sample(int dtype, const void *state, int n, uint64_t mask, uint64_t shots, uint64_t seed,
                          double *partials, double *offsets, uint64_t *d_out, cudaStream_t s) {
    const uint32_t chunk = (uint32_t)sample_chunk(n);
    const uint32_t P = (uint32_t)((1ull << n) / chunk);
    if (dtype == 0) k_sample_partials<float><<<P, 256, 0, s>>>(state, chunk, partials);
    else k_sample_partials<double><<<P, 256, 0, s>>>(state, chunk, partials);
    k_sample_scan<<<1, 1024, 0, s>>>(partials, P, offsets);
    if (shots) {
        const uint64_t blocks = std::min<uint64_t>((shots + 7) / 8, 152ull * 8);
        if (dtype == 0)
            k_sample_draw<float><<<(unsigned)blocks, 256, 0, s>>>(state, chunk, P, offsets, seed, shots, mask, d_out);
        else
            k_sample_draw<double><<<(unsigned)blocks, 256, 0, s>>>(state, chunk, P, offsets, seed, shots, mask, d_out);
    }
    return cudaGetLastError();
}

cudaError_t launch_tile_pass_multi(int dtype, int threads, int kmax, const TileArgs *d_descs,
                                   int n_desc, uint32_t total_ctas, int max_m, cudaStream_t s) {
    if (n_desc <= 0 || total_ctas == 0) return cudaSuccess;
    const size_t smem = tile_smem_bytes(dtype, max_m);
    if (kmax > 2) {
        if (dtype == 0) k_tile_pass_multi<float, 256, 5><<<total_ctas, 256, smem, s>>>(d_descs, n_desc);
        else k_tile_pass_multi<double, 256, 5><<<total_ctas, 256, smem, s>>>(d_descs, n_desc);
    } else if (dtype == 0) {
        if (threads == 512) k_tile_pass_multi<float, 512, 2><<<total_ctas, 512, smem, s>>>(d_descs, n_desc);
        else k_tile_pass_multi<float, 256, 2><<<total_ctas, 256, smem, s>>>(d_descs, n_desc);
    } else {
        if (threads == 512) k_tile_pass_multi<double, 512, 2><<<total_ctas, 512, smem, s>>>(d_descs, n_desc);
        else k_tile_pass_multi<double, 256, 2><<<total_ctas, 256, smem, s>>>(d_descs, n_desc);
    }
    return cudaGetLastError();
}

size_t tile_smem_bytes(int dtype, int m) {
    const size_t es = dtype == 0 ? 8 : 16;
    return (es << m) + es * kPassMats + sizeof(DevOp) * kPassOps;
}

cudaError_t launch_resident(int dtype, int kmax, const Instance &inst, cudaStream_t s) {
    const size_t smem = resident_smem_bytes(dtype, inst.n);
    if (kmax > 2) {
        if (dtype == 0) k_resident_one<float, 256, 5><<<1, 256, smem, s>>>(inst);
        else k_resident_one<double, 256, 5><<<1, 256, smem, s>>>(inst);
    } else {
        if (dtype == 0) k_resident_one<float, 256, 2><<<1, 256, smem, s>>>(inst);
        else k_resident_one<double, 256, 2><<<1, 256, smem, s>>>(inst);
    }
    return cudaGetLastError();
}

cudaError_t launch_resident_batch(int dtype, int kmax, const Instance *d_insts, int count,
                                  int max_n, cudaStream_t s) {
    if (count <= 0) return cudaSuccess;
    const size_t smem = resident_smem_bytes(dtype, max_n);
    if (kmax > 2) {
        if (dtype == 0) k_resident_batch<float, 256, 5><<<count, 256, smem, s>>>(d_insts, max_n);
        else k_resident_batch<double, 256, 5><<<count, 256, smem, s>>>(d_insts, max_n);
    } else {
        if (dtype == 0) k_resident_batch<float, 256, 2><<<count, 256, smem, s>>>(d_insts, max_n);
        else k_resident_batch<double, 256, 2><<<count, 256, smem, s>>>(d_insts, max_n);
    }
    return cudaGetLastError();
}

int prob_blocks(int n) {
    // chunks of >= 2048 amplitudes, at most 1024 blocks, a power of two
    int lg = n - 11;
    if (lg < 0) lg = 0;
    if (lg > 10) lg = 10;
    return 1 << lg;
}

cudaError_t launch_measure(int dtype, void *state, int n, const MeasArgs &a, double *partials,
                           MeasCtl *ctl, MeasRec *log, cudaStream_t s) {
    const int P = prob_blocks(n);
    if (dtype == 0) k_prob<float, true><<<P, kRedThreads, 0, s>>>(state, n, a, partials, ctl, log);
    else k_prob<double, true><<<P, kRedThreads, 0, s>>>(state, n, a, partials, ctl, log);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const uint64_t half = 1ull << (n - 1);
    uint64_t g = (half + 255) / 256;
    if (g > 4096) g = 4096;
    if (dtype == 0) k_collapse<float><<<(unsigned)g, 256, 0, s>>>(state, n, a.q, a.reset, ctl);
    else k_collapse<double><<<(unsigned)g, 256, 0, s>>>(state, n, a.q, a.reset, ctl);
    return cudaGetLastError();
}

cudaError_t launch_prob_only(int dtype, const void *state, int n, int q, double *partials,
                             MeasCtl *ctl, cudaStream_t s) {
    const int P = prob_blocks(n);
    MeasArgs a{};
    a.q = q;
    if (dtype == 0) k_prob<float, false><<<P, kRedThreads, 0, s>>>(state, n, a, partials, ctl, nullptr);
    else k_prob<double, false><<<P, kRedThreads, 0, s>>>(state, n, a, partials, ctl, nullptr);
    return cudaGetLastError();
}

cudaError_t launch_expect_batch(int dtype, const ExpectJob *d_jobs, int count, cudaStream_t s) {
    if (count <= 0) return cudaSuccess;
    if (dtype == 0) k_expect_batch<float><<<count, 256, 0, s>>>(d_jobs);
    else k_expect_batch<double><<<count, 256, 0, s>>>(d_jobs);
    return cudaGetLastError();
}

int expect_blocks(int n) {
    int lg = n - 12;
    if (lg < 0) lg = 0;
    if (lg > 8) lg = 8;
    return 1 << lg;
}

cudaError_t launch_expect(int dtype, const void *state, int n, const uint64_t *d_terms,
                          size_t n_terms, double *partials, double *d_out, cudaStream_t s) {
    if (n_terms == 0) return cudaSuccess;
    const int P = expect_blocks(n);
    size_t done = 0;
    while (done < n_terms) {  // grid.y <= 65535
        const size_t cnt = n_terms - done < 65535 ? n_terms - done : 65535;
        dim3 grid(P, (unsigned)cnt);
        if (dtype == 0) k_expect<float><<<grid, 256, 0, s>>>(state, n, d_terms + 3 * done, partials + done * P);
        else k_expect<double><<<grid, 256, 0, s>>>(state, n, d_terms + 3 * done, partials + done * P);
        done += cnt;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_expect_final<<<(unsigned)((n_terms + 255) / 256), 256, 0, s>>>(d_terms, n_terms, P, partials, d_out);
    return cudaGetLastError();
}

cudaError_t launch_set_basis(int dtype, void *state, int n, uint64_t index, cudaStream_t s) {
    const uint64_t N = 1ull << n;
    uint64_t g = (N + 255) / 256;
    if (g > 8192) g = 8192;
    if (dtype == 0) k_set_basis<float><<<(unsigned)g, 256, 0, s>>>(state, N, index);
    else k_set_basis<double><<<(unsigned)g, 256, 0, s>>>(state, N, index);
    return cudaGetLastError();
}

}  // namespace qsim
