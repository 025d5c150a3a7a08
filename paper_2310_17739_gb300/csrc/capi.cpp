// capi.cpp -- the C ABI of include/qsim.h: contexts, device buffers, program
// upload, launch sequencing, and the pipelined compile-and-launch of qsim_apply
// (host threads compile chunks of the gate stream while earlier chunks run).
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/qsim.h"
#include "compiler.h"
#include "kernels.h"

#include <cmath>

static_assert(qsim::kTilePassOps == qsim::kPassOps && qsim::kTilePassMats == qsim::kPassMats,
              "the compiler's per-pass limits must match the tile kernel's shared-memory slices");

using qsim::cd;
using qsim::Config;
using qsim::DevOp;
using qsim::HostProgram;
using qsim::MeasCtl;
using qsim::MeasRec;
using qsim::Pass;

namespace {

// Host image of one compiled chunk, ready for upload: DevOps + matrices in the
// state's dtype, plus the pass list the launcher walks.
struct Packed {
    std::vector<DevOp> ops;
    std::vector<unsigned char> mats;
    std::vector<Pass> passes;
    std::vector<uint64_t> bvec;  // tile bases (Pass::basis indexes it)
    int n = 0, m = 0;
    bool resident = false;
    uint64_t gates = 0, measurements = 0, fused = 0, dense_passes = 0;
    uint64_t hist[8] = {0, 0, 0, 0, 0, 0, 0, 0};
};

// Device image of one compiled chunk.
struct DevChunk {
    DevOp *d_ops = nullptr;
    size_t n_ops = 0;
    void *d_mats = nullptr;
    size_t mats_bytes = 0;
    std::vector<Pass> passes;
    std::vector<uint64_t> bvec;
    int m = 0;
    int kmax = 2;
    bool resident = false;
    uint64_t measurements = 0;
};

// Whether the 2^k x 2^k matrix at M (row-major) has at most one nonzero entry
// per row; if so perm gets that entry's column for row r at bits 2r..2r+1.
bool monomial(const cd *M, int k, uint16_t *perm) {
    const int D = 1 << k;
    uint16_t p = 0;
    for (int r = 0; r < D; r++) {
        int col = -1;
        for (int c = 0; c < D; c++) {
            if (M[r * D + c] == cd(0.0, 0.0)) continue;
            if (col >= 0) return false;
            col = c;
        }
        if (col > 0) p |= (uint16_t)(col << (2 * r));
    }
    *perm = p;
    return true;
}

void pack(const HostProgram &hp, qsim_dtype dt, bool allow_reg, Packed &pk) {
    pk.n = hp.n;
    pk.m = hp.m;
    pk.resident = hp.resident;
    pk.gates = hp.gates;
    pk.measurements = hp.measurements;
    std::memcpy(pk.hist, hp.hist, sizeof(pk.hist));
    const size_t es = dt == QSIM_C64 ? 8 : 16;
    pk.mats.resize(hp.pool.size() * es);
    if (dt == QSIM_C64) {
        float *f = reinterpret_cast<float *>(pk.mats.data());
        for (size_t i = 0; i < hp.pool.size(); i++) {
            f[2 * i] = (float)hp.pool[i].real();
            f[2 * i + 1] = (float)hp.pool[i].imag();
        }
    } else if (!hp.pool.empty()) {
        std::memcpy(pk.mats.data(), hp.pool.data(), hp.pool.size() * 16);
    }
    // Ops are re-emitted pass by pass in tile coordinates (see Pass): a dense
    // op's qubits become the tile bits of their unit vectors; a rotation
    // exp(-i theta P), P = i^y X^xm Z^zm (y = #Y), becomes its X mask's
    // coordinates xt, its Z mask's parities over the basis zt (bit j =
    // parity(zm & basis_j)) and over the tile origin zc (zm gathered from the
    // non-pivot positions, which the block index spreads x0 over), plus the
    // factor -i i^y = i^e folded into its coefficient (cos theta, W):
    //   a'_j = cos a_j + W (odd ? i : 1) (-1)^{parity(k & zm)} a_k,  k = j ^ xm,
    // with W = +-sin theta and odd = e & 1 in lq[4] bit 0.
    // A complex64 pass made only of rotations whose X coordinates have <= 5
    // bits is laid out in register segments (a kSegMarker op, then its
    // rotations, each with its X and Z coordinates over the segment's five
    // register positions in lq[4] bits 1..5 and lq[5]) for the register
    // tile kernel.
    pk.passes.clear();
    pk.ops.clear();
    pk.ops.reserve(hp.ops.size() + hp.passes.size() * 2);
    pk.bvec = hp.bvec;
    uint64_t fused = 0, dp = 0;
    const bool reg_dtype = dt == QSIM_C64 && !hp.resident && hp.m >= 10 && hp.m <= 14;
    auto set_coef = [&](uint64_t idx, double c, double w) {
        if (dt == QSIM_C64) {
            float *f = reinterpret_cast<float *>(pk.mats.data()) + 2 * idx;
            f[0] = (float)c;
            f[1] = (float)w;
        } else {
            double *f = reinterpret_cast<double *>(pk.mats.data()) + 2 * idx;
            f[0] = c;
            f[1] = w;
        }
    };
    // per-pass scratch, reused across passes (cleared before each use)
    std::vector<DevOp> body, cur;
    std::vector<float> tab, tvals;
    std::vector<size_t> cur_ix;
    std::vector<std::vector<uint32_t>> succ;
    std::vector<uint32_t> waits;
    std::vector<char> placed;
    struct OpSupport {
        uint64_t m, x, z;
        bool rot;
    };
    std::vector<OpSupport> sup;
    for (const Pass &src : hp.passes) {
        Pass p = src;
        p.first = pk.ops.size();
        if (src.ev) {
            const qsim::FOp &o = hp.ops[src.first];
            DevOp d;
            std::memset(&d, 0, sizeof(d));
            d.ev = o.ev;
            d.flags = o.flags;
            d.lq[0] = (uint8_t)o.q[0];
            pk.ops.push_back(d);
            p.count = 1;
            pk.passes.push_back(p);
            continue;
        }
        dp++;
        const int m = hp.resident ? hp.n : hp.m;
        uint64_t *B = pk.bvec.data() + src.basis;
        const uint64_t nonpiv = ~src.tile & (hp.n >= 64 ? ~0ull : ((1ull << hp.n) - 1));
        auto gather = [&](uint64_t v) {  // v's bits at the non-pivot positions, packed
            uint32_t r = 0;
            int j = 0;
            for (uint64_t b = nonpiv; b; b &= b - 1, j++) r |= (uint32_t)((v >> __builtin_ctzll(b)) & 1) << j;
            return r;
        };
        bool all_rot = true;
        bool regable = true;    // every op fits a register segment (rotation or dense k <= 2)
        bool has_dense = false;
        uint32_t mono_saved = 0;  // algorithmic flops per amplitude saved by monomial ops
        double gprod = 1.0;       // product of the cosines of the rotations in scaled form
        auto emit_body = [&]() {
            qsim::Subspace S;
            for (int j = 0; j < m; j++) S.add(B[j]);
            body.clear();
            all_rot = true;
            regable = true;
            has_dense = false;
            mono_saved = 0;
            gprod = 1.0;
            for (uint64_t i = src.first; i < src.first + src.count; i++) {
                const qsim::FOp &o = hp.ops[i];
                DevOp d;
                std::memset(&d, 0, sizeof(d));
                d.k = o.k;
                // the tile kernel indexes the pass's own coefficient slice; the
                // resident kernel walks the whole pool
                d.mat = (uint32_t)(hp.resident ? o.mat : o.mat - src.mat_first);
                if (o.pauli()) {
                    const uint32_t lx = S.coords(o.xm);
                    uint32_t lz = 0;
                    for (int j = 0; j < m; j++) lz |= (uint32_t)(__builtin_popcountll(o.zm & B[j]) & 1) << j;
                    const uint32_t zc = gather(o.zm);
                    d.lq[0] = (uint8_t)(lx & 0xff);
                    d.lq[1] = (uint8_t)(lx >> 8);
                    d.lq[2] = (uint8_t)(lz & 0xff);
                    d.lq[3] = (uint8_t)(lz >> 8);
                    // -i i^y, times i^g for a frame flush (whose cos is 0)
                    const int e = (__builtin_popcountll(o.xm & o.zm) + 3 + (o.flags & qsim::kPhaseMask)) & 3;
                    d.lq[4] = (uint8_t)(e & 1);
                    d.flags = (uint16_t)(zc & 0xffff);
                    d.pad = (uint16_t)(zc >> 16);
                    const cd cs = hp.pool[o.mat];
                    const double w = e >= 2 ? -cs.imag() : cs.imag();
                    // scaled form in tile passes (not in the resident kernel):
                    // a' = a + (W / cos) (...), the cosine applied at write-back;
                    // only while the running product stays >= 2^-40, so that the
                    // unscaled amplitudes cannot grow beyond 2^40
                    if (!hp.resident && std::fabs(cs.real()) >= 0.5 &&
                        std::fabs(gprod * cs.real()) >= 0x1p-40) {
                        set_coef(o.mat, cs.real(), w / cs.real());
                        d.lq[4] |= 2;
                        gprod *= cs.real();
                    } else {
                        set_coef(o.mat, cs.real(), w);
                    }
                    if (__builtin_popcount(lx) > 5) all_rot = regable = false;
                } else {
                    for (int j = 0; j < o.k; j++) d.lq[j] = (uint8_t)__builtin_ctz(S.coords(1ull << o.q[j]));
                    uint16_t perm = 0;
                    if (o.k <= 2 && monomial(hp.pool.data() + o.mat, o.k, &perm)) {
                        d.k = o.k == 1 ? qsim::kMono1 : qsim::kMono2;
                        d.flags = perm;
                        mono_saved += (8u << o.k) - 8u;
                    }
                    all_rot = false;
                    has_dense = true;
                    if (o.k > 2) regable = false;
                }
                body.push_back(d);
            }
        };
        emit_body();
        // register segments: a rotation-only pass over its gadget basis, or any
        // pass whose ops are rotations with <= 5 X coordinates and dense ops of
        // <= 2 qubits
        bool reg = allow_reg && reg_dtype && hp.n <= 32 && (src.gadget ? all_rot : regable);
        // the generic tile kernel wants the basis vectors after the leading
        // unit ones free of those low bits (whole 16-byte runs per row)
        auto reduce_basis = [&]() {
            int l = 0;
            while (l < m && B[l] == (1ull << l)) l++;
            const uint64_t low = l >= 64 ? ~0ull : ((1ull << l) - 1);
            for (int j = l; j < m; j++) B[j] &= ~low;
        };
        if (reg) {
            // scaled form: every cosine is >= 1/sqrt(2) after the Pauli frame
            double scale = 1.0;
            for (uint64_t i = src.first; i < src.first + src.count && reg; i++) {
                if (!hp.ops[i].pauli()) continue;
                const cd cs = hp.pool[hp.ops[i].mat];
                if (std::fabs(cs.real()) < 0.5) reg = false;
                scale *= cs.real();
                if (std::fabs(scale) < 0x1p-40) reg = false;  // unscaled amplitudes would grow beyond 2^40
            }
            if (reg) {
                for (uint64_t i = src.first; i < src.first + src.count; i++) {
                    const qsim::FOp &o = hp.ops[i];
                    if (!o.pauli()) continue;
                    const cd cs = hp.pool[o.mat];
                    const int e = (__builtin_popcountll(o.xm & o.zm) + 3 + (o.flags & qsim::kPhaseMask)) & 3;
                    const double w = e >= 2 ? -cs.imag() : cs.imag();
                    set_coef(o.mat, cs.real(), w / cs.real());
                }
                p.scale = (float)scale;
            }
        }
        if (!reg && src.gadget) {
            reduce_basis();
            emit_body();
        }
        fused += body.size();
        if (reg) {
            // greedy segments: grow the register set with each rotation's X
            // positions while it stays <= 5; fill it up with the highest free
            // positions (so that the lowest tile positions index threads)
            std::vector<std::pair<uint32_t, std::vector<DevOp>>> segs;
            tab.clear();  // the pass's coefficient tables (floats)
            const float *tvals_f = reinterpret_cast<const float *>(pk.mats.data());
            tvals.assign(src.mat_count, 0.0f);  // t of each rotation, by relative coefficient index
            for (uint32_t q = 0; q < src.mat_count; q++) tvals[q] = tvals_f[2 * (src.mat_first + q) + 1];
            uint32_t R = 0;
            cur.clear();
            cur_ix.clear();  // body index of each op of cur
            // tile positions an op needs in registers: a rotation's X
            // coordinates, a dense op's qubits
            auto need = [&](const DevOp &d) -> uint32_t {
                if (d.k == qsim::kPauli) return d.lq[0] | ((uint32_t)d.lq[1] << 8);
                const int k = (d.k == 1 || d.k == qsim::kMono1) ? 1 : 2;
                uint32_t r = 1u << d.lq[0];
                if (k == 2) r |= 1u << d.lq[1];
                return r;
            };
            auto close = [&]() {
                if (cur.empty()) return;
                for (int b = m - 1; b >= 0 && __builtin_popcount(R) < 5; b--) R |= 1u << b;
                int pos[5];
                for (int b = 0, j = 0; b < 32; b++)
                    if ((R >> b) & 1) pos[j++] = b;
                for (size_t ci = 0; ci < cur.size(); ci++) {
                    DevOp &d = cur[ci];
                    if (d.k != qsim::kPauli) {
                        // dense op: its slots, its matrix (local bit 0 <-> the lower slot)
                        const qsim::FOp &o = hp.ops[src.first + cur_ix[ci]];
                        const bool mono = d.k == qsim::kMono1 || d.k == qsim::kMono2;
                        const int k = (d.k == 1 || d.k == qsim::kMono1) ? 1 : 2, D = 1 << k;
                        int sl[2] = {0, 0};
                        for (int j = 0; j < k; j++)
                            for (int t = 0; t < 5; t++)
                                if (pos[t] == d.lq[j]) sl[j] = t;
                        const bool swap = k == 2 && sl[0] > sl[1];
                        auto sig = [&](int l) { return swap ? ((l & 1) << 1) | ((l >> 1) & 1) : l; };
                        cd M[16];
                        uint16_t perm = 0;
                        for (int r = 0; r < D; r++)
                            for (int c = 0; c < D; c++) M[sig(r) * D + sig(c)] = hp.pool[o.mat + (uint64_t)(r * D + c)];
                        if (mono)
                            for (int r = 0; r < D; r++)
                                perm |= (uint16_t)(sig((d.flags >> (2 * r)) & 3) << (2 * sig(r)));
                        const int s0 = std::min(sl[0], sl[1]), s1 = std::max(sl[0], sl[1]);
                        static const int pair_no[5][5] = {{-1, 0, 1, 2, 3}, {0, -1, 4, 5, 6}, {1, 4, -1, 7, 8},
                                                          {2, 5, 7, -1, 9}, {3, 6, 8, 9, -1}};
                        qsim::RegDense rd;
                        std::memset(&rd, 0, sizeof(rd));
                        rd.k = qsim::kDenseReg;
                        // a monomial C2 runs in one of three column patterns
                        // (diagonal, CX controlled by the lower or by the higher
                        // slot); any other runs as a dense C2 of the same matrix
                        int pat = -1;
                        if (mono && k == 2) pat = perm == 0xE4 ? 0 : perm == 0x6C ? 1 : perm == 0xB4 ? 2 : -1;
                        rd.sel = (uint8_t)(k == 1 ? (mono ? 15 : 0) + sl[0]
                                                  : (pat >= 0 ? 20 + 10 * pat : 5) + pair_no[s0][s1]);
                        rd.perm = perm;
                        rd.tab = (uint32_t)tab.size();
                        const size_t t0 = tab.size();
                        tab.resize(t0 + 2 * (size_t)(D * D));
                        for (int q = 0; q < D * D; q++) {
                            tab[t0 + 2 * q] = (float)M[q].real();
                            tab[t0 + 2 * q + 1] = (float)M[q].imag();
                        }
                        std::memcpy(&d, &rd, sizeof(d));
                        continue;
                    }
                    const uint32_t x = d.lq[0] | ((uint32_t)d.lq[1] << 8);
                    const uint32_t z = d.lq[2] | ((uint32_t)d.lq[3] << 8);
                    uint32_t xr = 0, zr = 0;
                    for (int j = 0; j < 5; j++) {
                        xr |= ((x >> pos[j]) & 1u) << j;
                        zr |= ((z >> pos[j]) & 1u) << j;
                    }
                    const float t = tvals[d.mat];
                    qsim::RegRot r;
                    std::memset(&r, 0, sizeof(r));
                    r.k = qsim::kPauli;
                    r.sel = (uint8_t)((d.lq[4] & 1) | (xr << 1));
                    r.zt = (uint16_t)z;
                    r.zc = d.flags | ((uint32_t)d.pad << 16);
                    r.tab = (uint32_t)tab.size();
                    // u over the pairs (slots for xr = 0), then negated
                    const int H = xr ? 31 - __builtin_clz(xr) : -1;
                    const int cnt = xr ? 16 : 32;
                    float u[32];
                    for (int q = 0; q < cnt; q++) {
                        const uint32_t j = H < 0 ? (uint32_t)q : (((uint32_t)q >> H) << (H + 1)) | ((uint32_t)q & ((1u << H) - 1));
                        u[q] = (__builtin_popcount(j & zr) & 1) ? -t : t;
                    }
                    const size_t t0 = tab.size();
                    tab.resize(t0 + 2 * (size_t)cnt);
                    for (int q = 0; q < cnt; q++) {
                        tab[t0 + q] = u[q];
                        tab[t0 + cnt + q] = -u[q];
                    }
                    std::memcpy(&d, &r, sizeof(d));
                }
                segs.emplace_back(R, cur);
                cur.clear();
                cur_ix.clear();
                R = 0;
            };
            // List scheduling over the pass's rotations: an op is ready once
            // every earlier op it does not commute with is placed; a segment
            // takes ready ops whose X coordinates it already holds first, then
            // the ready op that grows it least, and closes when none fits.
            const size_t K = body.size();
            if (succ.size() < K) succ.resize(K);  // succ[a]: later ops that must wait for op a
            for (size_t a = 0; a < K; a++) succ[a].clear();
            waits.assign(K, 0);
            // the pass's ops as (support, X, Z, is rotation): ops_commute on them
            sup.resize(K);
            for (size_t a = 0; a < K; a++) {
                const qsim::FOp &o = hp.ops[src.first + a];
                sup[a] = {o.mask(), o.xm, o.zm, o.pauli()};
            }
            for (size_t a = 0; a < K; a++)
                for (size_t b = a + 1; b < K; b++) {
                    const OpSupport &u = sup[a], &v = sup[b];
                    const bool commute = !(u.m & v.m) || (u.rot && v.rot && ((__builtin_popcountll(u.x & v.z) +
                                                                              __builtin_popcountll(u.z & v.x)) & 1) == 0);
                    if (!commute) {
                        succ[a].push_back((uint32_t)b);
                        waits[b]++;
                    }
                }
            placed.assign(K, 0);
            size_t left = K;
            while (left) {
                int best = -1, best_grow = 6;
                for (size_t a = 0; a < K; a++) {
                    if (placed[a] || waits[a]) continue;
                    const uint32_t x = need(body[a]);
                    const int grow = __builtin_popcount(x & ~R);
                    if (__builtin_popcount(R | x) <= 5 && grow < best_grow) {
                        best = (int)a;
                        best_grow = grow;
                        if (!grow) break;
                    }
                }
                if (best < 0) {  // nothing ready fits: a new segment
                    close();
                    continue;
                }
                R |= need(body[best]);
                cur.push_back(body[best]);
                cur_ix.push_back((size_t)best);
                placed[best] = 1;
                for (uint32_t b : succ[best]) waits[b]--;
                left--;
            }
            close();
            if (body.size() + segs.size() <= (size_t)qsim::kPassOps && tab.size() <= 2 * (size_t)qsim::kPassMats) {
                // the tables replace the pass's coefficient slice (appended)
                while (pk.mats.size() % 16) pk.mats.push_back(0);
                p.mat_first = pk.mats.size() / 8;
                p.mat_count = (uint32_t)((tab.size() + 1) / 2);
                const size_t off = pk.mats.size();
                pk.mats.resize(off + (size_t)p.mat_count * 8, 0);
                std::memcpy(pk.mats.data() + off, tab.data(), tab.size() * sizeof(float));
                for (auto &sg : segs) {
                    DevOp mk;
                    std::memset(&mk, 0, sizeof(mk));
                    mk.k = qsim::kSegMarker;
                    mk.flags = (uint16_t)sg.second.size();
                    for (int b = 0, j = 0; b < 32; b++)
                        if ((sg.first >> b) & 1) mk.lq[j++] = (uint8_t)b;
                    pk.ops.push_back(mk);
                    pk.ops.insert(pk.ops.end(), sg.second.begin(), sg.second.end());
                }
                p.reg = has_dense ? 2 : 1;
                p.count = (uint32_t)(pk.ops.size() - p.first);
                p.fpa -= std::min(p.fpa, mono_saved);
                pk.passes.push_back(p);
                continue;
            }
            // too many ops for one register-segment pass: the generic kernel
            // runs it, with plain (cos, W) coefficients over the reduced basis
            reduce_basis();
            emit_body();
            p.scale = 1.0f;
        }
        pk.ops.insert(pk.ops.end(), body.begin(), body.end());
        p.count = (uint32_t)(pk.ops.size() - p.first);
        p.fpa -= std::min(p.fpa, mono_saved);
        p.gscale = gprod;
        pk.passes.push_back(p);
    }
    pk.fused = fused;
    pk.dense_passes = dp;
}

struct Staging {
    void *host = nullptr;
    size_t bytes = 0;
    cudaEvent_t done = nullptr;
};

thread_local std::string g_err;

}  // namespace

struct qsim_ctx {
    int n = 0;
    qsim_dtype dtype = QSIM_C64;
    int device = 0;
    cudaStream_t stream = nullptr;
    qsim_alloc_fn alloc = nullptr;
    qsim_free_fn free_fn = nullptr;
    void *user = nullptr;
    void *state = nullptr;
    size_t state_bytes = 0;
    MeasCtl *ctl = nullptr;
    MeasRec *log = nullptr;
    size_t log_cap = 0;
    uint64_t log_n = 0;
    double *partials = nullptr;
    unsigned long long *tile_ctr = nullptr;  // persistent rotation passes: tile counter
    unsigned long long tile_base = 0;        // its value when the next such pass starts
    size_t partials_cap = 0;  // doubles
    uint64_t ordinal = 0;
    uint64_t seed = 0;
    double thr = 0.0;
    Config cfg;
    bool multi_state = false;  // a batch instance: its passes run in multi-state launches
    MeasCtl *h_ctl = nullptr;  // pinned readback of the control block
    std::vector<Staging> staging;
    std::string err;
    bool broken = false;
    // sampled tile-pass timing
    int prof_every = 0;
    uint64_t prof_launches = 0;
    size_t prof_used = 0;       // closed windows (event pairs)
    bool prof_open = false;     // a window's start event is recorded
    uint32_t prof_in_window = 0;
    uint64_t prof_sampled = 0;  // tile-pass launches inside closed windows
    double prof_flops = 0, prof_bytes = 0;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> prof_ev;
    // live programs compiled on this context (released and orphaned by qsim_destroy)
    std::vector<qsim_program *> programs;
    uint64_t cfg_gen = 0;                 // bumped by qsim_set_config (invalidates program graphs)
    cudaStream_t cap_stream = nullptr;    // private stream for graph capture (nothing runs on it)
    // graphs launched by qsim_apply, destroyed once the event after them has completed
    std::deque<std::pair<cudaEvent_t, std::vector<cudaGraphExec_t>>> graph_retire;
    cudaEvent_t sync_ev = nullptr;        // qsim_sync_timeout: recorded behind the enqueued work
};

// A run of consecutive tile passes of one chunk (no measurement between
// them), replayed as one CUDA graph launch once captured.
struct PassRun {
    size_t first = 0, end = 0;        // pass indices [first, end) in DevChunk::passes
    uint64_t launches = 0;            // tile-pass launches in it
    double flops = 0;                 // algorithmic flops of those launches
    cudaGraphExec_t exec = nullptr;
};

struct qsim_program {
    qsim_ctx *owner = nullptr;
    std::vector<DevChunk> chunks;
    qsim_program_info info{};
    // graph replay (qsim_config::graphs): per chunk, its runs of tile passes
    mutable uint64_t runs_done = 0;   // completed qsim_run calls
    mutable bool graphs_ready = false, graphs_failed = false;
    mutable uint64_t graph_gen = 0;   // ctx cfg_gen the graphs were captured under
    mutable std::vector<std::vector<PassRun>> runs;
};

namespace {

qsim_status fail(qsim_ctx *c, qsim_status s, const std::string &msg) {
    if (c) c->err = msg;
    g_err = msg;
    return s;
}

qsim_status cuda_fail(qsim_ctx *c, cudaError_t e, const char *what) {
    std::string msg = std::string(what) + ": " + cudaGetErrorString(e);
    if (c) c->broken = true;
    return fail(c, QSIM_E_CUDA, msg);
}

#define CK(expr, what)                                         \
    do {                                                       \
        cudaError_t e_ = (expr);                               \
        if (e_ != cudaSuccess) return cuda_fail(c, e_, what);  \
    } while (0)

void *dalloc(qsim_ctx *c, size_t bytes) {
    if (bytes == 0) bytes = 16;
    if (c->alloc) return c->alloc(bytes, c->stream, c->user);
    void *p = nullptr;
    if (cudaMallocAsync(&p, bytes, c->stream) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return p;
}

void dfree(qsim_ctx *c, void *p, size_t bytes) {
    if (!p) return;
    if (c->free_fn) c->free_fn(p, bytes, c->stream, c->user);
    else cudaFreeAsync(p, c->stream);
}

// A pinned staging buffer whose previous copy has completed.
Staging *get_staging(qsim_ctx *c, size_t bytes) {
    for (auto &s : c->staging)
        if (s.bytes >= bytes && cudaEventQuery(s.done) == cudaSuccess) return &s;
    cudaGetLastError();
    if (c->staging.size() >= 8) {  // bound pinned memory: wait for the oldest fitting one
        for (auto &s : c->staging)
            if (s.bytes >= bytes) {
                cudaEventSynchronize(s.done);
                return &s;
            }
    }
    Staging s;
    s.bytes = std::max(bytes, (size_t)1 << 20);
    if (cudaHostAlloc(&s.host, s.bytes, cudaHostAllocDefault) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (cudaEventCreateWithFlags(&s.done, cudaEventDisableTiming) != cudaSuccess) {
        cudaFreeHost(s.host);
        cudaGetLastError();
        return nullptr;
    }
    c->staging.push_back(s);
    return &c->staging.back();
}

// Stream-ordered upload of host bytes through a pinned staging buffer.
qsim_status upload(qsim_ctx *c, void *dst, const void *src, size_t bytes) {
    if (bytes == 0) return QSIM_OK;
    Staging *s = get_staging(c, bytes);
    if (!s) return fail(c, QSIM_E_OOM, "pinned staging allocation failed");
    std::memcpy(s->host, src, bytes);
    CK(cudaMemcpyAsync(dst, s->host, bytes, cudaMemcpyHostToDevice, c->stream), "upload");
    CK(cudaEventRecord(s->done, c->stream), "upload event");
    return QSIM_OK;
}

qsim_status ensure_log(qsim_ctx *c, uint64_t need) {
    if (need <= c->log_cap) return QSIM_OK;
    size_t cap = std::max<size_t>(c->log_cap * 2, 1024);
    while (cap < need) cap *= 2;
    MeasRec *nl = (MeasRec *)dalloc(c, cap * sizeof(MeasRec));
    if (!nl) return fail(c, QSIM_E_OOM, "measurement log allocation failed");
    if (c->log) {
        CK(cudaMemcpyAsync(nl, c->log, c->log_cap * sizeof(MeasRec), cudaMemcpyDeviceToDevice,
                           c->stream),
           "log grow");
        dfree(c, c->log, c->log_cap * sizeof(MeasRec));
    }
    c->log = nl;
    c->log_cap = cap;
    return QSIM_OK;
}

qsim_status ensure_partials(qsim_ctx *c, size_t doubles) {
    if (doubles <= c->partials_cap) return QSIM_OK;
    size_t cap = std::max<size_t>(c->partials_cap * 2, 4096);
    while (cap < doubles) cap *= 2;
    double *p = (double *)dalloc(c, cap * sizeof(double));
    if (!p) return fail(c, QSIM_E_OOM, "reduction scratch allocation failed");
    dfree(c, c->partials, c->partials_cap * sizeof(double));
    c->partials = p;
    c->partials_cap = cap;
    return QSIM_OK;
}

qsim_status check_usable(qsim_ctx *c) {
    if (!c) return fail(nullptr, QSIM_E_INVAL, "null context");
    if (c->broken) return fail(c, QSIM_E_STATE, "context unusable after an earlier CUDA error");
    cudaError_t e = cudaSetDevice(c->device);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaSetDevice");
    return QSIM_OK;
}

// Synchronise, read the control block, report deferred device failures.
void reap_graphs(qsim_ctx *c, bool wait);

qsim_status sync_read(qsim_ctx *c) {
    CK(cudaMemcpyAsync(c->h_ctl, c->ctl, sizeof(MeasCtl), cudaMemcpyDeviceToHost, c->stream),
       "control readback");
    CK(cudaStreamSynchronize(c->stream), "stream synchronize");
    reap_graphs(c, true);
    if (c->h_ctl->status == QSIM_E_ZEROPROB)
        return fail(c, QSIM_E_ZEROPROB,
                    "assertion-mode measurement #" + std::to_string(c->h_ctl->fail_log) +
                        " found P(0) <= threshold; later operations were skipped");
    return QSIM_OK;
}

qsim_status upload_chunk(qsim_ctx *c, const Packed &pk, DevChunk &dc) {
    dc.n_ops = pk.ops.size();
    dc.mats_bytes = pk.mats.size();
    dc.passes = pk.passes;
    dc.bvec = pk.bvec;
    dc.m = pk.m;
    dc.kmax = 1;  // largest dense op (Pauli rotations, hist[7], run in every variant)
    for (int k = 5; k >= 1; k--)
        if (pk.hist[k]) {
            dc.kmax = k;
            break;
        }
    dc.resident = pk.resident;
    dc.measurements = pk.measurements;
    dc.d_ops = (DevOp *)dalloc(c, std::max<size_t>(dc.n_ops, 1) * sizeof(DevOp));
    dc.d_mats = dalloc(c, std::max<size_t>(dc.mats_bytes, 16));
    if (!dc.d_ops || !dc.d_mats) {
        dfree(c, dc.d_ops, 0);
        dfree(c, dc.d_mats, 0);
        dc.d_ops = nullptr;
        dc.d_mats = nullptr;
        return fail(c, QSIM_E_OOM, "program allocation failed");
    }
    qsim_status s = upload(c, dc.d_ops, pk.ops.data(), dc.n_ops * sizeof(DevOp));
    if (s == QSIM_OK) s = upload(c, dc.d_mats, pk.mats.data(), dc.mats_bytes);
    return s;
}

void release_chunk(qsim_ctx *c, DevChunk &dc) {
    dfree(c, dc.d_ops, dc.n_ops * sizeof(DevOp));
    dfree(c, dc.d_mats, dc.mats_bytes);
    dc.d_ops = nullptr;
    dc.d_mats = nullptr;
}

qsim_status launch_measure(qsim_ctx *c, int q, int mode, int reset, uint64_t seed) {
    qsim_status s = ensure_log(c, c->log_n + 1);
    if (s != QSIM_OK) return s;
    s = ensure_partials(c, 2 * (size_t)qsim::prob_blocks(c->n));
    if (s != QSIM_OK) return s;
    qsim::MeasArgs a;
    std::memset(&a, 0, sizeof(a));
    a.q = q;
    a.mode = mode;
    a.reset = reset;
    a.seed = seed;
    a.ordinal = c->ordinal;
    a.log_idx = c->log_n;
    a.log_cap = c->log_cap;
    a.thr = c->thr;
    CK(qsim::launch_measure(c->dtype, c->state, c->n, a, c->partials, c->ctl, c->log, c->stream),
       "measure launch");
    c->ordinal++;
    c->log_n++;
    return QSIM_OK;
}

// Launch timing windows: up to kProfWindow consecutive tile-pass launches
// between two events, so that dependent launches inside a window still overlap.
constexpr int kProfWindow = 16;

cudaError_t profile_close(qsim_ctx *c) {
    if (!c->prof_open) return cudaSuccess;
    c->prof_open = false;
    const cudaError_t e = cudaEventRecord(c->prof_ev[c->prof_used].second, c->stream);
    c->prof_used++;
    c->prof_sampled += c->prof_in_window;
    return e;
}

// Threads per block of the generic tile pass: 512 for complex64 rotation
// passes (more warps in flight); dense C2 passes and complex128 keep 256 (their
// 512-thread builds are capped at 64 registers and lose more to spills than
// they gain).
int tile_threads(const qsim_ctx *c) {
    return c->cfg.threads ? c->cfg.threads : (c->dtype == QSIM_C64 && c->cfg.fusion == 2 ? 512 : 256);
}

// One tile pass (register-segment or generic) on stream s.
cudaError_t launch_tile(qsim_ctx *c, const DevChunk &dc, const Pass &p, int threads, cudaStream_t s) {
    const uint64_t *basis = dc.bvec.data() + p.basis;
    if (p.reg)
        return qsim::launch_rot_pass(c->state, c->n, dc.m, p.tile, basis, dc.d_ops + p.first, p.count, dc.d_mats,
                                     (uint32_t)p.mat_first, p.mat_count, p.scale, p.reg == 2, c->ctl, s);
    return qsim::launch_tile_pass(c->dtype, threads, dc.kmax, c->state, c->n, dc.m, p.tile, basis,
                                  dc.d_ops + p.first, p.count, dc.d_mats, (uint32_t)p.mat_first, p.mat_count,
                                  p.gscale, c->ctl, s);
}

qsim_status launch_chunk(qsim_ctx *c, const DevChunk &dc) {
    const int threads = tile_threads(c);
    if (dc.resident) {
        qsim_status s = ensure_log(c, c->log_n + dc.measurements);
        if (s != QSIM_OK) return s;
        qsim::Instance in;
        std::memset(&in, 0, sizeof(in));
        in.state = c->state;
        in.ops = dc.d_ops;
        in.mats = dc.d_mats;
        in.n_ops = dc.n_ops;
        in.seed = c->seed;
        in.ordinal0 = c->ordinal;
        in.log0 = c->log_n;
        in.log_cap = c->log_cap;
        in.ctl = c->ctl;
        in.log = c->log;
        in.thr = c->thr;
        in.n = c->n;
        if (dc.n_ops) CK(qsim::launch_resident(c->dtype, dc.kmax, in, c->stream), "resident launch");
        c->ordinal += dc.measurements;
        c->log_n += dc.measurements;
        return QSIM_OK;
    }
    for (const Pass &p : dc.passes) {
        if (p.ev) {
            CK(profile_close(c), "profile event");  // a window never spans a measurement
            qsim_status s = launch_measure(c, (int)p.q, p.flags, p.ev == qsim::EV_RESET, c->seed);
            if (s != QSIM_OK) return s;
            continue;
        }
        if (!p.count) continue;
        if (!c->prof_open && c->prof_every > 0 && c->prof_launches % (uint64_t)c->prof_every == 0 &&
            c->prof_used < c->prof_ev.size()) {
            CK(cudaEventRecord(c->prof_ev[c->prof_used].first, c->stream), "profile event");
            c->prof_open = true;
            c->prof_in_window = 0;
        }
        const uint64_t *pb = dc.bvec.data() + p.basis;
        if (p.reg == 1 && c->cfg.persistent && dc.m <= 13 && pb[0] == 1 && pb[1] == 2 && pb[2] == 4 && pb[3] == 8) {
            const uint64_t *basis = pb;
            if (!c->tile_ctr) {
                c->tile_ctr = (unsigned long long *)dalloc(c, sizeof(unsigned long long));
                if (!c->tile_ctr) return fail(c, QSIM_E_OOM, "tile counter allocation failed");
                CK(cudaMemsetAsync(c->tile_ctr, 0, sizeof(unsigned long long), c->stream), "tile counter");
                c->tile_base = 0;
            }
            uint32_t grid = 0;
            CK(qsim::launch_rot_pipe(c->state, c->n, dc.m, p.tile, basis, dc.d_ops + p.first, p.count,
                                     dc.d_mats, (uint32_t)p.mat_first, p.mat_count, p.scale, c->ctl,
                                     c->tile_ctr, c->tile_base, &grid, c->stream),
               "persistent rotation pass launch");
            c->tile_base += (1ull << (c->n - dc.m)) + grid;
        } else
            CK(launch_tile(c, dc, p, threads, c->stream), p.reg ? "rotation pass launch" : "tile pass launch");
        if (c->prof_open) {
            c->prof_in_window++;
            c->prof_flops += (double)p.fpa * (double)(1ull << c->n);
            c->prof_bytes += 2.0 * (double)c->state_bytes;
            if (c->prof_in_window >= (uint32_t)std::min(c->prof_every, kProfWindow))
                CK(profile_close(c), "profile event");
        }
        c->prof_launches++;
    }
    return QSIM_OK;
}

// ----------------------------------------------------------- graph replay --
// A compiled program replayed by qsim_run: every run of tile passes between two
// measurements is captured once as a CUDA graph (kernel nodes joined by the
// same programmatic dependencies as the stream launches) and then replayed
// with one graph launch, which saves the per-launch cost of stream launches.
constexpr uint64_t kGraphMaxPasses = 1ull << 21;
constexpr size_t kApplyGraphMin = 256;  // qsim_apply: chunks with fewer tile passes launch them directly

void destroy_graphs(qsim_ctx *c, const qsim_program *p) {
    bool any = false;
    for (auto &rs : p->runs)
        for (auto &r : rs) any = any || r.exec;
    if (any) cudaStreamSynchronize(c->stream);  // no launch of them may be pending
    for (auto &rs : p->runs)
        for (auto &r : rs)
            if (r.exec) cudaGraphExecDestroy(r.exec);
    p->runs.clear();
    p->graphs_ready = false;
    cudaGetLastError();
}

// Capture every run of tile passes of one chunk as a CUDA graph, on a private
// stream (capture enqueues nothing).  Returns false, with no graph left, if
// any capture or instantiation fails.
bool capture_chunk(qsim_ctx *c, const DevChunk &dc, std::vector<PassRun> &rs) {
    rs.clear();
    if (!c->cap_stream && cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
        c->cap_stream = nullptr;
        cudaGetLastError();
        return false;
    }
    const int threads = tile_threads(c);
    bool ok = true;
    for (size_t i = 0; ok && i < dc.passes.size();) {
        if (dc.passes[i].ev) {
            i++;
            continue;
        }
        PassRun r;
        r.first = i;
        for (; i < dc.passes.size() && !dc.passes[i].ev; i++)
            if (dc.passes[i].count) {
                r.launches++;
                r.flops += (double)dc.passes[i].fpa * (double)(1ull << c->n);
            }
        r.end = i;
        if (r.launches) {
            cudaGraph_t g = nullptr;
            cudaError_t e = cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal);
            if (e == cudaSuccess) {
                for (size_t k = r.first; e == cudaSuccess && k < r.end; k++)
                    if (dc.passes[k].count) e = launch_tile(c, dc, dc.passes[k], threads, c->cap_stream);
                const cudaError_t e2 = cudaStreamEndCapture(c->cap_stream, &g);
                if (e == cudaSuccess) e = e2;
            }
            if (e == cudaSuccess) e = cudaGraphInstantiate(&r.exec, g, 0);
            if (g) cudaGraphDestroy(g);
            if (e != cudaSuccess) {
                r.exec = nullptr;
                ok = false;
            }
        }
        rs.push_back(r);
    }
    if (!ok) {
        for (auto &r : rs)
            if (r.exec) cudaGraphExecDestroy(r.exec);
        rs.clear();
        cudaGetLastError();
    }
    return ok;
}

qsim_status build_graphs(qsim_ctx *c, const qsim_program *p) {
    destroy_graphs(c, p);
    uint64_t total = 0;
    for (const DevChunk &dc : p->chunks)
        if (!dc.resident)
            for (const Pass &ps : dc.passes) total += !ps.ev && ps.count;
    if (total > kGraphMaxPasses) {
        p->graphs_failed = true;
        return QSIM_OK;
    }
    p->runs.assign(p->chunks.size(), {});
    for (size_t ci = 0; ci < p->chunks.size(); ci++) {
        if (p->chunks[ci].resident) continue;
        if (!capture_chunk(c, p->chunks[ci], p->runs[ci])) {
            destroy_graphs(c, p);
            p->graphs_failed = true;
            return QSIM_OK;
        }
    }
    p->graphs_ready = true;
    return QSIM_OK;
}

// launch_chunk with each run of tile passes as one graph launch (a profiling
// window, when sampling is on, spans exactly one graph launch).
qsim_status run_chunk_graphs(qsim_ctx *c, const DevChunk &dc, const std::vector<PassRun> &rs) {
    size_t ri = 0;
    for (size_t i = 0; i < dc.passes.size();) {
        const Pass &ps = dc.passes[i];
        if (ps.ev) {
            CK(profile_close(c), "profile event");
            qsim_status s = launch_measure(c, (int)ps.q, ps.flags, ps.ev == qsim::EV_RESET, c->seed);
            if (s != QSIM_OK) return s;
            i++;
            continue;
        }
        if (ri >= rs.size() || rs[ri].first != i) return fail(c, QSIM_E_STATE, "graph runs out of step");
        const PassRun &r = rs[ri++];
        if (r.exec) {
            const bool win = c->prof_every > 0;
            if (win) CK(profile_close(c), "profile event");
            const bool open = win && c->prof_used < c->prof_ev.size();
            if (open) {
                CK(cudaEventRecord(c->prof_ev[c->prof_used].first, c->stream), "profile event");
                c->prof_open = true;
            }
            CK(cudaGraphLaunch(r.exec, c->stream), "graph launch");
            if (open) {
                c->prof_in_window = (uint32_t)r.launches;
                c->prof_flops += r.flops;
                c->prof_bytes += 2.0 * (double)c->state_bytes * (double)r.launches;
                CK(profile_close(c), "profile event");
            }
            c->prof_launches += r.launches;
        }
        i = r.end;
    }
    return QSIM_OK;
}

// A chunk launched once by qsim_apply: a long one runs as graph launches
// (capture and instantiation cost the host about what stream launches would;
// the device saves the per-launch cost); the graphs are destroyed once an event
// recorded after them has completed.
// Destroy the graphs of qsim_apply whose launches have completed (all of them,
// waiting, when `wait`).
void reap_graphs(qsim_ctx *c, bool wait) {
    while (!c->graph_retire.empty()) {
        auto &f = c->graph_retire.front();
        if (wait) cudaEventSynchronize(f.first);
        else if (cudaEventQuery(f.first) != cudaSuccess) break;
        for (cudaGraphExec_t g : f.second) cudaGraphExecDestroy(g);
        cudaEventDestroy(f.first);
        c->graph_retire.pop_front();
    }
    cudaGetLastError();  // cudaErrorNotReady from the query
}

qsim_status launch_chunk_once(qsim_ctx *c, const DevChunk &dc) {
    reap_graphs(c, false);
    size_t tile_passes = 0;
    for (const Pass &ps : dc.passes) tile_passes += !ps.ev && ps.count;
    std::vector<PassRun> rs;
    if (c->cfg.graphs == 2 || c->cfg.persistent || dc.resident || tile_passes < kApplyGraphMin ||
        !capture_chunk(c, dc, rs))
        return launch_chunk(c, dc);
    const qsim_status st = run_chunk_graphs(c, dc, rs);
    std::vector<cudaGraphExec_t> ex;
    for (auto &r : rs)
        if (r.exec) ex.push_back(r.exec);
    cudaEvent_t ev = nullptr;
    if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) == cudaSuccess &&
        cudaEventRecord(ev, c->stream) == cudaSuccess) {
        c->graph_retire.emplace_back(ev, std::move(ex));
    } else {  // no event: wait for the stream before destroying them
        cudaGetLastError();
        if (ev) cudaEventDestroy(ev);
        cudaStreamSynchronize(c->stream);
        for (cudaGraphExec_t g : ex) cudaGraphExecDestroy(g);
    }
    return st;
}

// Chunk boundaries over ng gate records: chunk_gates each when set; by default
// 2^16 gates first, doubling up to 2^20, so that the device starts on the first
// chunk while the host still compiles the later, larger ones.
std::vector<size_t> chunk_bounds(const qsim_ctx *c, size_t ng) {
    std::vector<size_t> b{0};
    size_t C = c->cfg.chunk_gates > 0 ? (size_t)c->cfg.chunk_gates : ((size_t)1 << 16);
    const size_t cap = c->cfg.chunk_gates > 0 ? C : ((size_t)1 << 20);
    while (b.back() < ng) {
        b.push_back(std::min(ng, b.back() + C));
        C = std::min(cap, 2 * C);
    }
    return b;
}

// Register-segment layout for rotation passes: single-state launches with the
// default thread count only (the multi-state kernel runs the generic pass).
bool allow_reg(const qsim_ctx *c) { return c->cfg.threads == 0; }

int compile_threads(const qsim_ctx *c) {
    if (c->cfg.compile_threads > 0) return c->cfg.compile_threads;
    unsigned h = std::thread::hardware_concurrency();
    return (int)std::max(1u, std::min(h > 1 ? h - 1 : 1u, 32u));
}

// Compile chunks [0, nchunks) on worker threads and hand them, in order, to
// `sink`.  At most `ahead` chunks are compiled but not yet consumed.
template <class Sink>
qsim_status compile_chunks(qsim_ctx *c, const qsim_gate *g, size_t ng, const double *mats,
                           size_t nm, Sink sink) {
    const std::vector<size_t> bounds = chunk_bounds(c, ng);
    const size_t nchunks = bounds.size() - 1;
    if (nchunks <= 1) {
        HostProgram hp;
        qsim::compile(c->n, c->dtype, c->cfg, g, ng, mats, nm, hp);
        Packed pk;
        pack(hp, c->dtype, allow_reg(c), pk);
        return sink(pk);
    }
    const int T = std::min<int>(compile_threads(c), (int)nchunks);
    const size_t ahead = (size_t)T * 2;
    std::vector<std::unique_ptr<Packed>> slots(nchunks);
    std::mutex mu;
    std::condition_variable cv;
    std::atomic<size_t> next{0};
    size_t consumed = 0;
    bool stop = false;
    auto worker = [&]() {
        for (;;) {
            size_t i;
            {
                std::unique_lock<std::mutex> lk(mu);
                cv.wait(lk, [&] { return stop || next.load() < consumed + ahead || next.load() >= nchunks; });
                if (stop || next.load() >= nchunks) return;
                i = next++;
            }
            const size_t b = bounds[i], e = bounds[i + 1];
            HostProgram hp;
            qsim::compile(c->n, c->dtype, c->cfg, g + b, e - b, mats, nm, hp);
            auto pk = std::make_unique<Packed>();
            pack(hp, c->dtype, allow_reg(c), *pk);
            {
                std::lock_guard<std::mutex> lk(mu);
                slots[i] = std::move(pk);
            }
            cv.notify_all();
        }
    };
    std::vector<std::thread> th;
    for (int t = 0; t < T; t++) th.emplace_back(worker);
    qsim_status st = QSIM_OK;
    for (size_t i = 0; i < nchunks; i++) {
        std::unique_ptr<Packed> pk;
        {
            std::unique_lock<std::mutex> lk(mu);
            cv.wait(lk, [&] { return slots[i] != nullptr; });
            pk = std::move(slots[i]);
            consumed = i + 1;
        }
        cv.notify_all();
        st = sink(*pk);
        if (st != QSIM_OK) break;
    }
    {
        std::lock_guard<std::mutex> lk(mu);
        stop = true;
    }
    cv.notify_all();
    for (auto &t : th) t.join();
    return st;
}

void accumulate(qsim_program_info &info, const Packed &pk, size_t dev_bytes) {
    info.gates += pk.gates;
    info.fused_ops += pk.fused;
    info.passes += pk.dense_passes;
    info.measurements += pk.measurements;
    info.device_bytes += dev_bytes;
    for (int k = 0; k < 8; k++) info.op_hist[k] += pk.hist[k];
}

// Every field of a caller's qsim_config in its documented range (n = 0: the
// state size is not known yet, so the tile_bits / n relation is not checked).
bool check_config(const qsim_config *cfg, qsim_dtype dtype, int n, std::string &err) {
    if (cfg->struct_size != sizeof(qsim_config)) {
        err = "qsim_config.struct_size is " + std::to_string(cfg->struct_size) + ", this library's qsim_config has " +
              std::to_string(sizeof(qsim_config)) + " bytes (initialise it with qsim_config_init)";
        return false;
    }
    const int mx = qsim::max_resident_bits(dtype);
    if (cfg->fusion < 0 || cfg->fusion > 2) err = "fusion must be 0, 1 or 2";
    else if (cfg->k_max != 0 && (cfg->k_max < 2 || cfg->k_max > 5)) err = "k_max must be 0 or in [2, 5]";
    else if (cfg->tile_bits < 0 || cfg->tile_bits > mx) err = "tile_bits out of range for this dtype";
    else if (n > 0 && cfg->tile_bits > 0 && cfg->tile_bits < n && cfg->tile_bits < 6)
        err = "tile_bits must be >= 6 unless it covers the whole state";
    else if (cfg->threads != 0 && cfg->threads != 256 && cfg->threads != 512) err = "threads must be 0, 256 or 512";
    else if (cfg->chunk_gates < 0 || cfg->lookahead < 0 || cfg->compile_threads < 0) err = "negative size";
    else if (cfg->persistent != 0 && cfg->persistent != 1) err = "persistent must be 0 or 1";
    else if (cfg->graphs < 0 || cfg->graphs > 2) err = "graphs must be 0, 1 or 2";
    else if (cfg->forced_low < 0 || cfg->forced_low > (dtype == QSIM_C64 ? 4 : 3))
        err = dtype == QSIM_C64 ? "forced_low must be in [0, 4] for complex64" : "forced_low must be in [0, 3] for complex128";
    else return true;
    return false;
}

}  // namespace

extern "C" {

const char *qsim_status_string(qsim_status s) {
    switch (s) {
        case QSIM_OK: return "ok";
        case QSIM_E_INVAL: return "invalid argument";
        case QSIM_E_OOM: return "out of memory";
        case QSIM_E_CUDA: return "CUDA error";
        case QSIM_E_ZEROPROB: return "assertion failed: P(0) <= threshold";
        case QSIM_E_TIMEOUT: return "timeout";
        case QSIM_E_STATE: return "context unusable";
        case QSIM_E_CANCELED: return "request cancelled";
    }
    return "unknown status";
}

const char *qsim_last_error(const qsim_ctx *c) { return c ? c->err.c_str() : g_err.c_str(); }

qsim_status qsim_create(int n, qsim_dtype dtype, void *stream, qsim_alloc_fn alloc,
                        qsim_free_fn free_fn, void *user, qsim_ctx **out) {
    if (!out) return fail(nullptr, QSIM_E_INVAL, "out is NULL");
    *out = nullptr;
    if (n < 1 || n > 34) return fail(nullptr, QSIM_E_INVAL, "n_qubits must be in [1, 34]");
    if (dtype != QSIM_C64 && dtype != QSIM_C128) return fail(nullptr, QSIM_E_INVAL, "bad dtype");
    if ((alloc == nullptr) != (free_fn == nullptr))
        return fail(nullptr, QSIM_E_INVAL, "alloc and free must be given together");
    static std::once_flag once;
    static cudaError_t setup_err = cudaSuccess;
    std::call_once(once, [] { setup_err = qsim::setup_kernels(); });
    if (setup_err != cudaSuccess)
        return fail(nullptr, QSIM_E_CUDA, std::string("kernel setup: ") + cudaGetErrorString(setup_err));
    auto c = std::make_unique<qsim_ctx>();
    c->n = n;
    c->dtype = dtype;
    c->stream = (cudaStream_t)stream;
    c->alloc = alloc;
    c->free_fn = free_fn;
    c->user = user;
    if (cudaGetDevice(&c->device) != cudaSuccess) {
        cudaGetLastError();
        return fail(nullptr, QSIM_E_CUDA, "no CUDA device");
    }
    c->state_bytes = (size_t)(dtype == QSIM_C64 ? 8 : 16) << n;
    c->state = dalloc(c.get(), c->state_bytes);
    if (!c->state) return fail(nullptr, QSIM_E_OOM, "state allocation failed");
    c->ctl = (MeasCtl *)dalloc(c.get(), sizeof(MeasCtl));
    if (cudaMallocHost((void **)&c->h_ctl, sizeof(MeasCtl)) != cudaSuccess) {
        cudaGetLastError();
        c->h_ctl = nullptr;
    }
    if (!c->ctl || !c->h_ctl) {
        dfree(c.get(), c->state, c->state_bytes);
        dfree(c.get(), c->ctl, sizeof(MeasCtl));
        if (c->h_ctl) cudaFreeHost(c->h_ctl);
        return fail(nullptr, QSIM_E_OOM, "control block allocation failed");
    }
    qsim_status s = qsim_reset_state(c.get());
    if (s != QSIM_OK) {
        qsim_destroy(c.release());
        return s;
    }
    *out = c.release();
    return QSIM_OK;
}

qsim_status qsim_destroy(qsim_ctx *c) {
    if (!c) return QSIM_OK;
    cudaSetDevice(c->device);
    // programs still alive release their device buffers now and become orphans
    reap_graphs(c, true);
    for (qsim_program *p : c->programs) {
        destroy_graphs(c, p);
        for (auto &dc : p->chunks) release_chunk(c, dc);
        p->owner = nullptr;
    }
    c->programs.clear();
    dfree(c, c->state, c->state_bytes);
    dfree(c, c->ctl, sizeof(MeasCtl));
    dfree(c, c->log, c->log_cap * sizeof(MeasRec));
    dfree(c, c->partials, c->partials_cap * sizeof(double));
    dfree(c, c->tile_ctr, sizeof(unsigned long long));
    cudaStreamSynchronize(c->stream);
    for (auto &s : c->staging) {
        cudaEventDestroy(s.done);
        cudaFreeHost(s.host);
    }
    if (c->h_ctl) cudaFreeHost(c->h_ctl);
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    if (c->sync_ev) cudaEventDestroy(c->sync_ev);
    for (auto &e : c->prof_ev) {
        cudaEventDestroy(e.first);
        cudaEventDestroy(e.second);
    }
    cudaGetLastError();
    delete c;
    return QSIM_OK;
}

qsim_status qsim_set_stream(qsim_ctx *c, void *stream) {
    qsim_status s = check_usable(c);
    if (s != QSIM_OK) return s;
    // order the new stream after everything enqueued on the old one
    CK(cudaStreamSynchronize(c->stream), "stream synchronize");
    c->stream = (cudaStream_t)stream;
    return QSIM_OK;
}

void qsim_config_init(qsim_config *cfg) {
    if (!cfg) return;
    qsim::config_to(Config(), cfg);
}

qsim_status qsim_set_config(qsim_ctx *c, const qsim_config *cfg) {
    if (!c || !cfg) return fail(c, QSIM_E_INVAL, "null argument");
    std::string err;
    if (!check_config(cfg, c->dtype, c->n, err)) return fail(c, QSIM_E_INVAL, err);
    c->cfg = qsim::config_from(cfg);
    c->cfg_gen++;
    return QSIM_OK;
}

qsim_status qsim_get_config(const qsim_ctx *c, qsim_config *cfg) {
    if (!c || !cfg) return QSIM_E_INVAL;
    qsim::config_to(c->cfg, cfg);
    return QSIM_OK;
}

qsim_status qsim_set_seed(qsim_ctx *c, uint64_t seed) {
    if (!c) return fail(nullptr, QSIM_E_INVAL, "null context");
    c->seed = seed;
    return QSIM_OK;
}

qsim_status qsim_set_assert_threshold(qsim_ctx *c, double thr) {
    if (!c) return fail(nullptr, QSIM_E_INVAL, "null context");
    if (!(thr >= 0.0 && thr < 1.0)) return fail(c, QSIM_E_INVAL, "threshold must be in [0, 1)");
    c->thr = thr;
    return QSIM_OK;
}

qsim_status qsim_apply(qsim_ctx *c, const qsim_gate *g, size_t ng, const double *mats, size_t nm) {
    qsim_status s = check_usable(c);
    if (s != QSIM_OK) return s;
    if (ng && !g) return fail(c, QSIM_E_INVAL, "gates is NULL");
    std::string err;
    if (!qsim::validate(c->n, g, ng, mats, nm, err)) return fail(c, QSIM_E_INVAL, err);
    return compile_chunks(c, g, ng, mats, nm, [&](const Packed &pk) -> qsim_status {
        DevChunk dc;
        qsim_status st = upload_chunk(c, pk, dc);
        if (st == QSIM_OK) st = launch_chunk_once(c, dc);
        release_chunk(c, dc);  // stream-ordered: freed after the launches above
        return st;
    });
}

qsim_status qsim_compile(qsim_ctx *c, const qsim_gate *g, size_t ng, const double *mats, size_t nm,
                         qsim_program **out) {
    qsim_status s = check_usable(c);
    if (s != QSIM_OK) return s;
    if (!out) return fail(c, QSIM_E_INVAL, "out is NULL");
    *out = nullptr;
    if (ng && !g) return fail(c, QSIM_E_INVAL, "gates is NULL");
    std::string err;
    if (!qsim::validate(c->n, g, ng, mats, nm, err)) return fail(c, QSIM_E_INVAL, err);
    auto prog = std::make_unique<qsim_program>();
    prog->owner = c;
    s = compile_chunks(c, g, ng, mats, nm, [&](const Packed &pk) -> qsim_status {
        DevChunk dc;
        qsim_status st = upload_chunk(c, pk, dc);
        if (st != QSIM_OK) {
            release_chunk(c, dc);
            return st;
        }
        accumulate(prog->info, pk, dc.n_ops * sizeof(DevOp) + dc.mats_bytes);
        prog->chunks.push_back(std::move(dc));
        return QSIM_OK;
    });
    if (s != QSIM_OK) {
        qsim_program_free(prog.release());
        return s;
    }
    c->programs.push_back(prog.get());
    *out = prog.release();
    return QSIM_OK;
}

qsim_status qsim_run(qsim_ctx *c, const qsim_program *p) {
    qsim_status s = check_usable(c);
    if (s != QSIM_OK) return s;
    if (!p || p->owner != c) return fail(c, QSIM_E_INVAL, "program does not belong to this context");
    const int mode = c->cfg.graphs;
    const bool want = mode != 2 && !c->cfg.persistent && !p->graphs_failed && (p->runs_done >= 1 || mode == 1);
    if (!want && p->graphs_ready) destroy_graphs(c, p);
    if (want && (!p->graphs_ready || p->graph_gen != c->cfg_gen)) {
        s = build_graphs(c, p);
        if (s != QSIM_OK) return s;
        p->graph_gen = c->cfg_gen;
    }
    const bool use = want && p->graphs_ready;
    for (size_t ci = 0; ci < p->chunks.size(); ci++) {
        const DevChunk &dc = p->chunks[ci];
        s = use && !dc.resident ? run_chunk_graphs(c, dc, p->runs[ci]) : launch_chunk(c, dc);
        if (s != QSIM_OK) return s;
    }
    p->runs_done++;
    return QSIM_OK;
}

qsim_status qsim_program_get_info(const qsim_program *p, qsim_program_info *info) {
    if (!p || !info) return QSIM_E_INVAL;
    *info = p->info;
    return QSIM_OK;
}

qsim_status qsim_program_free(qsim_program *p) {
    if (!p) return QSIM_OK;
    if (p->owner) {  // an orphan (its context destroyed) holds no device memory any more
        qsim_ctx *c = p->owner;
        cudaSetDevice(c->device);
        destroy_graphs(c, p);
        for (auto &dc : p->chunks) release_chunk(c, dc);
        c->programs.erase(std::remove(c->programs.begin(), c->programs.end(), p), c->programs.end());
    }
    delete p;
    return QSIM_OK;
}

qsim_status qsim_measure(qsim_ctx *c, int qubit, uint64_t seed, int mode, int *outcome, double *prob) {
    qsim_status s = check_usable(c);
    if (s != QSIM_OK) return s;
    if (qubit < 0 || qubit >= c->n) return fail(c, QSIM_E_INVAL, "qubit out of range");
    if (mode != 0 && mode != 1) return fail(c, QSIM_E_INVAL, "mode must be 0 or 1");
    const uint64_t idx = c->log_n;
    s = launch_measure(c, qubit, mode, 0, seed);
    if (s != QSIM_OK) return s;
    if (!outcome && !prob) return QSIM_OK;
    MeasRec rec;
    CK(cudaMemcpyAsync(c->h_ctl, c->ctl, sizeof(MeasCtl), cudaMemcpyDeviceToHost, c->stream), "readback");
    CK(cudaMemcpyAsync(&rec, c->log + idx, sizeof(rec), cudaMemcpyDeviceToHost, c->stream), "readback");
    CK(cudaStreamSynchronize(c->stream), "stream synchronize");
    if (c->h_ctl->status == QSIM_E_ZEROPROB) {
        if (c->h_ctl->fail_log == idx) {
            if (outcome) *outcome = -1;
            if (prob) *prob = rec.prob;
            return fail(c, QSIM_E_ZEROPROB, "assertion failed: P(0) <= threshold");
        }
        return fail(c, QSIM_E_ZEROPROB, "an earlier assertion-mode measurement failed");
    }
    if (outcome) *outcome = rec.outcome;
    if (prob) *prob = rec.prob;
    return QSIM_OK;
}

qsim_status qsim_prob(qsim_ctx *c, int qubit, double *p0, double *p1) {
    qsim_status s = check_usable(c);
    if (s != QSIM_OK) return s;
    if (qubit < 0 || qubit >= c->n) return fail(c, QSIM_E_INVAL, "qubit out of range");
    s = ensure_partials(c, 2 * (size_t)qsim::prob_blocks(c->n));
    if (s != QSIM_OK) return s;
    CK(qsim::launch_prob_only(c->dtype, c->state, c->n, qubit, c->partials, c->ctl, c->stream), "prob launch");
    s = sync_read(c);
    if (s != QSIM_OK) return s;
    if (p0) *p0 = c->h_ctl->p0;
    if (p1) *p1 = c->h_ctl->p1;
    return QSIM_OK;
}

qsim_status qsim_outcomes(qsim_ctx *c, int32_t *outcomes, double *probs, size_t cap, size_t *n_total) {
    qsim_status s = check_usable(c);
    if (s != QSIM_OK) return s;
    CK(cudaStreamSynchronize(c->stream), "stream synchronize");
    const size_t avail = std::min<uint64_t>(c->log_n, c->log_cap);
    if (n_total) *n_total = avail;
    const size_t k = std::min(avail, cap);
    if (k) {
        std::vector<MeasRec> recs(k);
        CK(cudaMemcpy(recs.data(), c->log, k * sizeof(MeasRec), cudaMemcpyDeviceToHost), "log readback");
        for (size_t i = 0; i < k; i++) {
            if (outcomes) outcomes[i] = recs[i].outcome;
            if (probs) probs[i] = recs[i].prob;
        }
    }
    return sync_read(c) == QSIM_E_CUDA ? QSIM_E_CUDA : QSIM_OK;
}

qsim_status qsim_success_prob(qsim_ctx *c, double *p) {
    qsim_status s = check_usable(c);
    if (s != QSIM_OK) return s;
    if (!p) return fail(c, QSIM_E_INVAL, "p is NULL");
    s = sync_read(c);
    *p = c->h_ctl->success;
    return s;
}

qsim_status qsim_expect(qsim_ctx *c, const qsim_pauli_term *t, size_t nt, double *out) {
    qsim_status s = check_usable(c);
    if (s != QSIM_OK) return s;
    if (nt == 0) return QSIM_OK;
    if (!t || !out) return fail(c, QSIM_E_INVAL, "null terms or out");
    const uint64_t full = c->n >= 64 ? ~0ull : ((1ull << c->n) - 1ull);
    for (size_t i = 0; i < nt; i++)
        if ((t[i].x_mask | t[i].z_mask) & ~full) return fail(c, QSIM_E_INVAL, "Pauli term beyond n qubits");
    const int P = qsim::expect_blocks(c->n);
    s = ensure_partials(c, (size_t)P * nt);
    if (s != QSIM_OK) return s;
    const size_t tb = nt * 3 * sizeof(uint64_t);
    uint64_t *d_terms = (uint64_t *)dalloc(c, tb);
    double *d_out = (double *)dalloc(c, nt * sizeof(double));
    if (!d_terms || !d_out) {
        dfree(c, d_terms, tb);
        dfree(c, d_out, nt * sizeof(double));
        return fail(c, QSIM_E_OOM, "expectation buffers");
    }
    static_assert(sizeof(qsim_pauli_term) == 24, "term layout");
    s = upload(c, d_terms, t, tb);
    if (s == QSIM_OK) {
        cudaError_t e = qsim::launch_expect(c->dtype, c->state, c->n, d_terms, nt, c->partials, d_out, c->stream);
        if (e != cudaSuccess) s = cuda_fail(c, e, "expect launch");
    }
    if (s == QSIM_OK) {
        cudaError_t e = cudaMemcpyAsync(out, d_out, nt * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
        if (e != cudaSuccess) s = cuda_fail(c, e, "expect readback");
    }
    dfree(c, d_terms, tb);
    dfree(c, d_out, nt * sizeof(double));
    if (s != QSIM_OK) return s;
    return sync_read(c);
}

qsim_status qsim_sample(qsim_ctx *c, uint64_t qubit_mask, uint64_t shots, uint64_t seed, uint64_t *out) {
    qsim_status s = check_usable(c);
    if (s != QSIM_OK) return s;
    const uint64_t full = c->n >= 64 ? ~0ull : ((1ull << c->n) - 1ull);
    if (qubit_mask & ~full) return fail(c, QSIM_E_INVAL, "qubit mask beyond n qubits");
    if (shots && !out) return fail(c, QSIM_E_INVAL, "null out");
    if (shots > (1ull << 40)) return fail(c, QSIM_E_INVAL, "too many shots");
    const uint64_t P = (1ull << c->n) / (uint64_t)qsim::sample_chunk(c->n);
    const size_t pb = (size_t)P * sizeof(double), ob = (size_t)(P + 1) * sizeof(double);
    const size_t sb = (size_t)std::max<uint64_t>(shots, 1) * sizeof(uint64_t);
    double *d_part = (double *)dalloc(c, pb);
    double *d_off = (double *)dalloc(c, ob);
    uint64_t *d_out = (uint64_t *)dalloc(c, sb);
    if (!d_part || !d_off || !d_out) {
        dfree(c, d_part, pb);
        dfree(c, d_off, ob);
        dfree(c, d_out, sb);
        return fail(c, QSIM_E_OOM, "sampling buffers");
    }
    cudaError_t e = qsim::launch_sample(c->dtype, c->state, c->n, qubit_mask, shots, seed, d_part, d_off, d_out,
                                        c->stream);
    if (e != cudaSuccess) s = cuda_fail(c, e, "sample launch");
    if (s == QSIM_OK && shots) {
        e = cudaMemcpyAsync(out, d_out, (size_t)shots * sizeof(uint64_t), cudaMemcpyDeviceToHost, c->stream);
        if (e != cudaSuccess) s = cuda_fail(c, e, "sample readback");
    }
    dfree(c, d_part, pb);
    dfree(c, d_off, ob);
    dfree(c, d_out, sb);
    if (s != QSIM_OK) return s;
    return sync_read(c);
}

qsim_status qsim_state(qsim_ctx *c, void *dst, size_t bytes, int dst_is_device) {
    qsim_status s = check_usable(c);
    if (s != QSIM_OK) return s;
    if (!dst || bytes != c->state_bytes) return fail(c, QSIM_E_INVAL, "dst NULL or size mismatch");
    CK(cudaMemcpyAsync(dst, c->state, bytes, dst_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                       c->stream),
       "state copy");
    CK(cudaStreamSynchronize(c->stream), "stream synchronize");
    return QSIM_OK;
}

qsim_status qsim_set_state(qsim_ctx *c, const void *src, size_t bytes, int src_is_device) {
    qsim_status s = check_usable(c);
    if (s != QSIM_OK) return s;
    if (!src || bytes != c->state_bytes) return fail(c, QSIM_E_INVAL, "src NULL or size mismatch");
    CK(cudaMemcpyAsync(c->state, src, bytes, src_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                       c->stream),
       "state copy");
    CK(cudaMemsetAsync(&c->ctl->status, 0, sizeof(int32_t), c->stream), "status clear");
    if (!src_is_device) CK(cudaStreamSynchronize(c->stream), "stream synchronize");
    return QSIM_OK;
}

qsim_status qsim_reset_state(qsim_ctx *c) {
    if (!c) return fail(nullptr, QSIM_E_INVAL, "null context");
    if (c->broken) return fail(c, QSIM_E_STATE, "context unusable after an earlier CUDA error");
    CK(cudaSetDevice(c->device), "cudaSetDevice");
    CK(qsim::launch_set_basis(c->dtype, c->state, c->n, 0, c->stream), "state reset");
    MeasCtl init;
    std::memset(&init, 0, sizeof(init));
    init.success = 1.0;
    *c->h_ctl = init;
    CK(cudaMemcpyAsync(c->ctl, c->h_ctl, sizeof(MeasCtl), cudaMemcpyHostToDevice, c->stream), "control reset");
    CK(cudaStreamSynchronize(c->stream), "stream synchronize");
    c->ordinal = 0;
    c->log_n = 0;
    return QSIM_OK;
}

qsim_status qsim_get_draw_ordinal(const qsim_ctx *c, uint64_t *k) {
    if (!c || !k) return QSIM_E_INVAL;
    *k = c->ordinal;
    return QSIM_OK;
}

qsim_status qsim_set_draw_ordinal(qsim_ctx *c, uint64_t k) {
    if (!c) return fail(nullptr, QSIM_E_INVAL, "null context");
    c->ordinal = k;
    return QSIM_OK;
}

qsim_status qsim_state_ptr(qsim_ctx *c, void **dptr, size_t *bytes) {
    if (!c || !dptr) return fail(c, QSIM_E_INVAL, "null argument");
    *dptr = c->state;
    if (bytes) *bytes = c->state_bytes;
    return QSIM_OK;
}

qsim_status qsim_sync(qsim_ctx *c) {
    qsim_status s = check_usable(c);
    if (s != QSIM_OK) return s;
    return sync_read(c);
}

qsim_status qsim_sync_timeout(qsim_ctx *c, double seconds) {
    qsim_status s = check_usable(c);
    if (s != QSIM_OK) return s;
    if (!(seconds >= 0)) return fail(c, QSIM_E_INVAL, "seconds must be >= 0");
    if (!c->sync_ev) CK(cudaEventCreateWithFlags(&c->sync_ev, cudaEventDisableTiming), "event create");
    CK(cudaEventRecord(c->sync_ev, c->stream), "event record");
    const double t_end = std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count() +
                         seconds;
    for (;;) {
        const cudaError_t e = cudaEventQuery(c->sync_ev);
        if (e == cudaSuccess) break;
        if (e != cudaErrorNotReady) return cuda_fail(c, e, "event query");
        const double now = std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
        if (now >= t_end)
            return fail(c, QSIM_E_TIMEOUT, "the enqueued work had not completed after " + std::to_string(seconds) +
                                               " s (it keeps running)");
        std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
    cudaGetLastError();  // cudaErrorNotReady from the queries
    return sync_read(c);  // completed: reads the control block without waiting
}

qsim_status qsim_profile_start(qsim_ctx *c, int every) {
    qsim_status s = check_usable(c);
    if (s != QSIM_OK) return s;
    if (every < 0) return fail(c, QSIM_E_INVAL, "every must be >= 0");
    CK(cudaStreamSynchronize(c->stream), "stream synchronize");
    const size_t cap = 8192;
    while (every > 0 && c->prof_ev.size() < cap) {
        cudaEvent_t a, b;
        CK(cudaEventCreate(&a), "event create");
        CK(cudaEventCreate(&b), "event create");
        c->prof_ev.emplace_back(a, b);
    }
    c->prof_every = every;
    c->prof_launches = 0;
    c->prof_used = 0;
    c->prof_open = false;
    c->prof_in_window = 0;
    c->prof_sampled = 0;
    c->prof_flops = c->prof_bytes = 0;
    return QSIM_OK;
}

qsim_status qsim_profile_read(qsim_ctx *c, double *ms, uint64_t *n_sampled, double *flops, double *bytes,
                              uint64_t *n_launches) {
    qsim_status s = check_usable(c);
    if (s != QSIM_OK) return s;
    CK(profile_close(c), "profile event");
    CK(cudaStreamSynchronize(c->stream), "stream synchronize");
    double tot = 0;
    for (size_t i = 0; i < c->prof_used; i++) {
        float t = 0;
        CK(cudaEventElapsedTime(&t, c->prof_ev[i].first, c->prof_ev[i].second), "event elapsed");
        tot += t;
    }
    if (ms) *ms = tot;
    if (n_sampled) *n_sampled = c->prof_sampled;
    if (flops) *flops = c->prof_flops;
    if (bytes) *bytes = c->prof_bytes;
    if (n_launches) *n_launches = c->prof_launches;
    return QSIM_OK;
}

// ----------------------------------------------------- host-only inspection --
qsim_status qsim_fuse(int n, qsim_dtype dtype, const qsim_gate *g, size_t ng, const double *mats,
                      size_t nm, const qsim_config *cfg, uint8_t *out_k, uint32_t *out_q,
                      uint64_t *out_mat, size_t cap_ops, double *out_mats, size_t cap_mat_doubles,
                      size_t *n_ops, size_t *n_mat_doubles) {
    if (n < 1 || n > 34 || (ng && !g)) return fail(nullptr, QSIM_E_INVAL, "bad arguments");
    if (dtype != QSIM_C64 && dtype != QSIM_C128) return fail(nullptr, QSIM_E_INVAL, "bad dtype");
    std::string err;
    if (cfg && !check_config(cfg, dtype, n, err)) return fail(nullptr, QSIM_E_INVAL, err);
    if (!qsim::validate(n, g, ng, mats, nm, err)) return fail(nullptr, QSIM_E_INVAL, err);
    HostProgram hp;
    qsim::compile(n, dtype, qsim::config_from(cfg), g, ng, mats, nm, hp);
    if (n_ops) *n_ops = hp.ops.size();
    if (n_mat_doubles) *n_mat_doubles = hp.pool.size() * 2;
    if (hp.ops.size() > cap_ops || hp.pool.size() * 2 > cap_mat_doubles)
        return fail(nullptr, QSIM_E_INVAL, "output capacity too small");
    for (size_t i = 0; i < hp.ops.size(); i++) {
        const qsim::FOp &o = hp.ops[i];
        out_k[i] = o.k;
        for (int j = 0; j < 6; j++) out_q[6 * i + j] = 0;
        if (o.pauli()) {
            out_q[6 * i] = (uint32_t)o.xm;
            out_q[6 * i + 1] = (uint32_t)(o.xm >> 32);
            out_q[6 * i + 2] = (uint32_t)o.zm;
            out_q[6 * i + 3] = (uint32_t)(o.zm >> 32);
            out_q[6 * i + 4] = o.flags;
            out_mat[i] = o.mat * 2;
        } else if (o.k) {
            for (int j = 0; j < o.k; j++) out_q[6 * i + j] = o.q[j];
            out_mat[i] = o.mat * 2;
        } else {
            out_q[6 * i] = o.q[0];
            out_q[6 * i + 1] = o.ev == qsim::EV_MEASURE ? QSIM_OP_MEASURE
                               : o.ev == qsim::EV_RESET  ? QSIM_OP_RESET
                                                         : QSIM_OP_BARRIER;
            out_q[6 * i + 2] = o.flags;
            out_mat[i] = 0;
        }
    }
    if (!hp.pool.empty()) std::memcpy(out_mats, hp.pool.data(), hp.pool.size() * 16);
    return QSIM_OK;
}

qsim_status qsim_schedule(int n, qsim_dtype dtype, const qsim_gate *g, size_t ng, const double *mats,
                          size_t nm, const qsim_config *cfg, uint64_t *out_tile, uint64_t *out_first,
                          uint32_t *out_count, uint64_t *out_basis, size_t cap, size_t *n_passes) {
    if (n < 1 || n > 34 || (ng && !g)) return fail(nullptr, QSIM_E_INVAL, "bad arguments");
    if (dtype != QSIM_C64 && dtype != QSIM_C128) return fail(nullptr, QSIM_E_INVAL, "bad dtype");
    std::string err;
    if (cfg && !check_config(cfg, dtype, n, err)) return fail(nullptr, QSIM_E_INVAL, err);
    if (!qsim::validate(n, g, ng, mats, nm, err)) return fail(nullptr, QSIM_E_INVAL, err);
    HostProgram hp;
    qsim::compile(n, dtype, qsim::config_from(cfg), g, ng, mats, nm, hp);
    if (n_passes) *n_passes = hp.passes.size();
    if (hp.passes.size() > cap) return fail(nullptr, QSIM_E_INVAL, "output capacity too small");
    for (size_t i = 0; i < hp.passes.size(); i++) {
        out_tile[i] = hp.passes[i].ev ? 0 : hp.passes[i].tile;
        out_first[i] = hp.passes[i].first;
        out_count[i] = hp.passes[i].count;
        if (out_basis) {
            for (int j = 0; j < 16; j++) out_basis[16 * i + j] = 0;
            if (!hp.passes[i].ev)
                for (int j = 0; j < (hp.resident ? hp.n : hp.m); j++)
                    out_basis[16 * i + j] = hp.bvec[hp.passes[i].basis + j];
        }
    }
    return QSIM_OK;
}

}  // extern "C"

// ------------------------------------------------------------------ batches --
// A batch is a set of ordinary contexts (one per instance: state, control
// block, log) plus the launch plan, all on the batch stream: instances that fit
// one block's shared memory run together in one resident launch per (width,
// op size) group; the others advance in lockstep, pass k of all of them in one
// multi-state tile launch.
struct qsim_batch {
    int count = 0;
    qsim_dtype dtype = QSIM_C64;
    cudaStream_t stream = nullptr;
    std::vector<qsim_ctx *> inst;
    std::vector<std::vector<DevChunk>> prog;
    std::vector<char> resident;
    qsim_ctx *aux = nullptr;        // staging and scratch on the batch stream
    qsim::Instance *d_insts = nullptr;
    size_t insts_cap = 0;
    MeasCtl *h_init = nullptr;      // pinned cleared control block
    std::string err;
    // run replay: after one eager run (which makes every allocation), the next
    // run is captured into a CUDA graph and later runs replay it with one launch;
    // compiling, reconfiguring or reseeding any instance drops the graph
    // wide (tiled) instances advance in lockstep: step k runs pass k of every
    // one of them in one multi-state launch (events as per-instance launches)
    struct Step {
        size_t first = 0;       // generic passes: tiled_descs[first, first + count)
        int count = 0;
        uint32_t ctas = 0;
        int max_m = 1, kmax = 1;
        struct RegGroup {       // register-segment passes of one tile size
            size_t first = 0;
            int count = 0;
            uint32_t ctas = 0;
            int m = 0;
            bool dense = false;
        };
        std::vector<RegGroup> reg;
        std::vector<std::pair<int, Pass>> events;  // (instance, event pass)
    };
    bool plan_valid = false;
    std::vector<qsim::TileArgs> tiled_descs;
    std::vector<Step> steps;
    qsim::TileArgs *d_descs = nullptr;
    size_t descs_cap = 0;
    int eager_runs = 0;
    std::vector<uint64_t> meas_after;  // log records per instance after one run
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t graph_exec = nullptr;
    void drop_graph() {
        plan_valid = false;
        if (graph_exec) cudaGraphExecDestroy(graph_exec);
        if (graph) cudaGraphDestroy(graph);
        graph_exec = nullptr;
        graph = nullptr;
        eager_runs = 0;
    }
};

namespace {

qsim_status bfail(qsim_batch *b, qsim_status s, const std::string &msg) {
    if (b) b->err = msg;
    g_err = msg;
    return s;
}

// |0...0> and a cleared control block, enqueued on the context's stream.
qsim_status reset_async(qsim_ctx *c, const MeasCtl *h_init) {
    CK(qsim::launch_set_basis(c->dtype, c->state, c->n, 0, c->stream), "state reset");
    CK(cudaMemcpyAsync(c->ctl, h_init, sizeof(MeasCtl), cudaMemcpyHostToDevice, c->stream),
       "control reset");
    c->ordinal = 0;
    c->log_n = 0;
    return QSIM_OK;
}

void release_instance_program(qsim_batch *b, int i) {
    for (auto &dc : b->prog[i]) release_chunk(b->inst[i], dc);
    b->prog[i].clear();
}

}  // namespace

extern "C" {

qsim_status qsim_batch_destroy(qsim_batch *b) {
    if (!b) return QSIM_OK;
    cudaStreamSynchronize(b->stream);
    b->drop_graph();
    for (int i = 0; i < b->count; i++) {
        if (b->inst[i]) {
            release_instance_program(b, i);
            qsim_destroy(b->inst[i]);
        }
    }
    if (b->aux) {
        dfree(b->aux, b->d_insts, b->insts_cap * sizeof(qsim::Instance));
        dfree(b->aux, b->d_descs, b->descs_cap * sizeof(qsim::TileArgs));
        qsim_destroy(b->aux);
    }
    if (b->h_init) cudaFreeHost(b->h_init);
    cudaGetLastError();
    delete b;
    return QSIM_OK;
}

qsim_status qsim_batch_create(int count, const int32_t *n_qubits, qsim_dtype dtype, void *stream,
                              qsim_alloc_fn alloc, qsim_free_fn free_fn, void *user, qsim_batch **out) {
    if (!out) return fail(nullptr, QSIM_E_INVAL, "out is NULL");
    *out = nullptr;
    if (count <= 0 || !n_qubits) return fail(nullptr, QSIM_E_INVAL, "count must be > 0 with n_qubits given");
    for (int i = 0; i < count; i++)
        if (n_qubits[i] < 1 || n_qubits[i] > 34) return fail(nullptr, QSIM_E_INVAL, "n_qubits must be in [1, 34]");
    auto b = std::make_unique<qsim_batch>();
    b->count = count;
    b->dtype = dtype;
    b->stream = (cudaStream_t)stream;
    b->inst.assign(count, nullptr);
    b->prog.resize(count);
    b->resident.assign(count, 0);
    qsim_status s = qsim_create(1, dtype, stream, alloc, free_fn, user, &b->aux);
    if (s != QSIM_OK) return s;
    if (cudaMallocHost((void **)&b->h_init, sizeof(MeasCtl)) != cudaSuccess) {
        cudaGetLastError();
        qsim_batch_destroy(b.release());
        return fail(nullptr, QSIM_E_OOM, "batch host resources");
    }
    std::memset(b->h_init, 0, sizeof(MeasCtl));
    b->h_init->success = 1.0;
    const int mx = qsim::max_resident_bits(dtype);
    for (int i = 0; i < count; i++) {
        const int n = n_qubits[i];
        s = qsim_create(n, dtype, stream, alloc, free_fn, user, &b->inst[i]);
        if (s == QSIM_OK) b->inst[i]->multi_state = true;
        if (s != QSIM_OK) {
            qsim_batch_destroy(b.release());
            return s;
        }
        if (n <= mx) {
            b->resident[i] = 1;
            b->inst[i]->cfg.tile_bits = n;  // the whole state in one block
        }
    }
    *out = b.release();
    return QSIM_OK;
}

qsim_status qsim_batch_set_config(qsim_batch *b, const qsim_config *cfg) {
    if (!b || !cfg) return bfail(b, QSIM_E_INVAL, "null argument");
    if (cfg->struct_size != sizeof(qsim_config))  // before copying the caller's struct
        return bfail(b, QSIM_E_INVAL, "qsim_config.struct_size does not match this library (use qsim_config_init)");
    b->drop_graph();
    for (int i = 0; i < b->count; i++) {
        qsim_config c2 = *cfg;
        if (b->resident[i]) c2.tile_bits = b->inst[i]->n;  // residency is fixed at create
        qsim_status s = qsim_set_config(b->inst[i], &c2);
        if (s != QSIM_OK) return bfail(b, s, b->inst[i]->err);
    }
    return QSIM_OK;
}

qsim_status qsim_batch_set_instance_config(qsim_batch *b, int index, const qsim_config *cfg) {
    if (!b || !cfg || index < 0 || index >= b->count) return bfail(b, QSIM_E_INVAL, "bad batch index or null config");
    if (cfg->struct_size != sizeof(qsim_config))
        return bfail(b, QSIM_E_INVAL, "qsim_config.struct_size does not match this library (use qsim_config_init)");
    b->drop_graph();
    qsim_config c2 = *cfg;
    if (b->resident[index]) c2.tile_bits = b->inst[index]->n;  // residency is fixed at create
    qsim_status s = qsim_set_config(b->inst[index], &c2);
    return s == QSIM_OK ? QSIM_OK : bfail(b, s, b->inst[index]->err);
}

qsim_status qsim_batch_set_seeds(qsim_batch *b, const uint64_t *seeds) {
    if (!b || !seeds) return bfail(b, QSIM_E_INVAL, "null argument");
    b->drop_graph();
    for (int i = 0; i < b->count; i++) b->inst[i]->seed = seeds[i];
    return QSIM_OK;
}

qsim_status qsim_batch_compile(qsim_batch *b, int index, const qsim_gate *g, size_t ng,
                               const double *mats, size_t nm) {
    if (!b || index < 0 || index >= b->count) return bfail(b, QSIM_E_INVAL, "bad batch index");
    qsim_ctx *c = b->inst[index];
    if (ng && !g) return bfail(b, QSIM_E_INVAL, "gates is NULL");
    std::string err;
    if (!qsim::validate(c->n, g, ng, mats, nm, err)) return bfail(b, QSIM_E_INVAL, err);
    b->drop_graph();
    release_instance_program(b, index);
    // programs live on the batch stream (aux): uploaded before, freed after, every run
    auto sink = [&](const Packed &pk) -> qsim_status {
        DevChunk dc;
        qsim_status st = upload_chunk(b->aux, pk, dc);
        if (st != QSIM_OK) {
            release_chunk(b->aux, dc);
            return st;
        }
        b->prog[index].push_back(std::move(dc));
        return QSIM_OK;
    };
    qsim_status s;
    if (b->resident[index]) {  // the resident kernel walks one contiguous program
        HostProgram hp;
        qsim::compile(c->n, c->dtype, c->cfg, g, ng, mats, nm, hp);
        Packed pk;
        pack(hp, c->dtype, false, pk);
        s = sink(pk);
    } else {
        s = compile_chunks(c, g, ng, mats, nm, sink);
    }
    if (s != QSIM_OK) {
        release_instance_program(b, index);
        return bfail(b, s, b->aux->err);
    }
    return QSIM_OK;
}

qsim_status qsim_batch_compile_many(qsim_batch *b, int count, const int32_t *indices,
                                    const qsim_gate *const *gates, const size_t *n_gates,
                                    const double *const *mats, const size_t *n_mats, int threads) {
    if (!b || count < 0) return bfail(b, QSIM_E_INVAL, "bad batch or count");
    if (count && (!indices || !gates || !n_gates)) return bfail(b, QSIM_E_INVAL, "null argument");
    for (int k = 0; k < count; k++) {
        const int i = indices[k];
        if (i < 0 || i >= b->count) return bfail(b, QSIM_E_INVAL, "bad batch index");
        if (n_gates[k] && !gates[k]) return bfail(b, QSIM_E_INVAL, "gates is NULL");
        std::string err;
        if (!qsim::validate(b->inst[i]->n, gates[k], n_gates[k], mats ? mats[k] : nullptr, n_mats ? n_mats[k] : 0,
                            err))
            return bfail(b, QSIM_E_INVAL, err);
    }
    // host compilation of every program on worker threads (the same chunks as
    // qsim_batch_compile), then the uploads in order on the batch stream
    std::vector<std::vector<Packed>> packed((size_t)count);
    std::atomic<int> next{0};
    auto worker = [&]() {
        for (int k = next++; k < count; k = next++) {
            const int i = indices[k];
            qsim_ctx *c = b->inst[i];
            const double *mk = mats ? mats[k] : nullptr;
            const size_t nmk = n_mats ? n_mats[k] : 0;
            std::vector<size_t> bounds;
            if (!b->resident[i]) bounds = chunk_bounds(c, n_gates[k]);
            if (bounds.size() <= 2) bounds = {0, n_gates[k]};  // one program, as compile_chunks
            for (size_t j = 0; j + 1 < bounds.size(); j++) {
                const size_t lo = bounds[j], hi = bounds[j + 1];
                HostProgram hp;
                qsim::compile(c->n, c->dtype, c->cfg, gates[k] + lo, hi - lo, mk, nmk, hp);
                packed[k].emplace_back();
                pack(hp, c->dtype, b->resident[i] ? false : allow_reg(c), packed[k].back());
            }
        }
    };
    const int T = std::max(1, std::min(threads > 0 ? threads : compile_threads(b->aux), count));
    std::vector<std::thread> th;
    for (int t = 1; t < T; t++) th.emplace_back(worker);
    worker();
    for (auto &t : th) t.join();
    b->drop_graph();
    for (int k = 0; k < count; k++) {
        const int i = indices[k];
        release_instance_program(b, i);
        for (const Packed &pk : packed[k]) {
            DevChunk dc;
            qsim_status st = upload_chunk(b->aux, pk, dc);
            if (st != QSIM_OK) {
                release_chunk(b->aux, dc);
                release_instance_program(b, i);
                return bfail(b, st, b->aux->err);
            }
            b->prog[i].push_back(std::move(dc));
        }
        std::vector<Packed>().swap(packed[k]);
    }
    return QSIM_OK;
}

}  // extern "C"

namespace {

// Lockstep plan of the wide instances: step k holds pass k of each of them.
// May only allocate/upload when `may_upload` (an eager run).
qsim_status build_tiled_plan(qsim_batch *b, bool may_upload) {
    qsim_ctx *c = b->aux;
    b->tiled_descs.clear();
    b->steps.clear();
    // step k holds pass k of every wide instance
    struct Item {
        int i;
        const DevChunk *dc;
        const Pass *p;
    };
    std::vector<std::vector<Item>> per;
    for (int i = 0; i < b->count; i++) {
        if (b->resident[i]) continue;
        size_t k = 0;
        for (const DevChunk &dc : b->prog[i])
            for (const Pass &p : dc.passes) {
                if (!p.ev && !p.count) continue;
                if (per.size() <= k) per.resize(k + 1);
                per[k].push_back({i, &dc, &p});
                k++;
            }
    }
    b->steps.resize(per.size());
    for (size_t k = 0; k < per.size(); k++) {
        auto &st = b->steps[k];
        // the generic passes of the step (one multi-state launch), then its
        // register-segment passes grouped by (tile size, dense ops)
        st.first = b->tiled_descs.size();
        uint32_t ctas = 0;
        std::map<std::pair<int, int>, std::vector<qsim::TileArgs>> regs;
        for (const Item &it : per[k]) {
            if (it.p->ev) {
                st.events.emplace_back(it.i, *it.p);
                continue;
            }
            qsim_ctx *ic = b->inst[it.i];
            const DevChunk &dc = *it.dc;
            const Pass &p = *it.p;
            qsim::TileArgs a;
            if (!qsim::make_tile_args(b->dtype, ic->state, ic->n, dc.m, p.tile, dc.bvec.data() + p.basis,
                                      dc.d_ops + p.first, p.count, dc.d_mats, (uint32_t)p.mat_first, p.mat_count,
                                      ic->ctl, &a))
                return bfail(b, QSIM_E_INVAL, "pass does not fit the tile kernels");
            if (p.reg) {
                a.scale = p.scale;
                regs[std::make_pair(dc.m, p.reg == 2 ? 1 : 0)].push_back(a);
                continue;
            }
            if (!qsim::generic_tile_ok(a)) return bfail(b, QSIM_E_INVAL, "pass does not fit the tile kernel");
            a.wscale = p.gscale;
            a.cta_first = ctas;
            ctas += 1u << (a.n - a.m);
            st.max_m = std::max(st.max_m, a.m);
            st.kmax = std::max(st.kmax, std::max(dc.kmax, 1));
            b->tiled_descs.push_back(a);
            st.count++;
        }
        st.ctas = ctas;
        for (auto &g : regs) {
            qsim_batch::Step::RegGroup rg;
            rg.first = b->tiled_descs.size();
            rg.count = (int)g.second.size();
            rg.m = g.first.first;
            rg.dense = g.first.second != 0;
            uint32_t rc = 0;
            for (auto &a : g.second) {
                a.cta_first = rc;
                rc += 1u << (a.n - a.m);
                b->tiled_descs.push_back(a);
            }
            rg.ctas = rc;
            st.reg.push_back(rg);
        }
    }
    if (!b->tiled_descs.empty()) {
        if (!may_upload) return bfail(b, QSIM_E_STATE, "batch plan changed during capture");
        const size_t need = b->tiled_descs.size();
        if (need > b->descs_cap) {
            dfree(c, b->d_descs, b->descs_cap * sizeof(qsim::TileArgs));
            b->descs_cap = need;
            b->d_descs = (qsim::TileArgs *)dalloc(c, need * sizeof(qsim::TileArgs));
            if (!b->d_descs) {
                b->descs_cap = 0;
                return bfail(b, QSIM_E_OOM, "multi-state pass table");
            }
        }
        qsim_status s = upload(c, b->d_descs, b->tiled_descs.data(), need * sizeof(qsim::TileArgs));
        if (s != QSIM_OK) return bfail(b, s, c->err);
    }
    b->plan_valid = true;
    return QSIM_OK;
}

// Enqueue one run of every instance.  upload_table: (re)build and upload the
// resident instances' table (eager runs); a captured run reuses the table.
qsim_status enqueue_run(qsim_batch *b, bool upload_table) {
    qsim_ctx *c = b->aux;
    // resident instances, grouped by (width, largest op) so that each launch
    // sizes its shared memory for its own width
    std::vector<qsim::Instance> insts;
    std::vector<std::pair<std::pair<int, int>, size_t>> groups;  // ((n, kmax), first)
    std::vector<int> order;
    for (int i = 0; i < b->count; i++)
        if (b->resident[i]) order.push_back(i);
    auto kmax_of = [&](int i) { return b->prog[i].empty() ? 1 : b->prog[i][0].kmax; };
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
        const int nx = b->inst[x]->n, ny = b->inst[y]->n;
        return nx != ny ? nx < ny : (kmax_of(x) > 2) < (kmax_of(y) > 2);
    });
    for (int i : order) {
        qsim_ctx *ic = b->inst[i];
        const DevChunk *dc = b->prog[i].empty() ? nullptr : &b->prog[i][0];
        const uint64_t meas = dc ? dc->measurements : 0;
        qsim_status s = ensure_log(ic, meas);
        if (s != QSIM_OK) return bfail(b, s, ic->err);
        qsim::Instance in;
        std::memset(&in, 0, sizeof(in));
        in.state = ic->state;
        in.ops = dc ? dc->d_ops : nullptr;
        in.mats = dc ? dc->d_mats : nullptr;
        in.n_ops = dc ? dc->n_ops : 0;
        in.seed = ic->seed;
        in.log_cap = ic->log_cap;
        in.ctl = ic->ctl;
        in.log = ic->log;
        in.thr = ic->thr;
        in.n = ic->n;
        in.flags = qsim::kInstInit;
        const std::pair<int, int> key(ic->n, kmax_of(i) > 2 ? 5 : 2);
        if (groups.empty() || groups.back().first != key) groups.emplace_back(key, insts.size());
        insts.push_back(in);
        ic->ordinal = meas;
        ic->log_n = meas;
    }
    if (!insts.empty() && upload_table) {
        if (insts.size() > b->insts_cap) {
            dfree(c, b->d_insts, b->insts_cap * sizeof(qsim::Instance));
            b->insts_cap = std::max(insts.size(), (size_t)64);
            b->d_insts = (qsim::Instance *)dalloc(c, b->insts_cap * sizeof(qsim::Instance));
            if (!b->d_insts) {
                b->insts_cap = 0;
                return bfail(b, QSIM_E_OOM, "instance table");
            }
        }
        qsim_status s = upload(c, b->d_insts, insts.data(), insts.size() * sizeof(qsim::Instance));
        if (s != QSIM_OK) return bfail(b, s, c->err);
    }
    if (!insts.empty()) {
        for (size_t gi = 0; gi < groups.size(); gi++) {
            const size_t first = groups[gi].second;
            const size_t last = gi + 1 < groups.size() ? groups[gi + 1].second : insts.size();
            CK(qsim::launch_resident_batch(b->dtype, groups[gi].first.second, b->d_insts + first,
                                           (int)(last - first), groups[gi].first.first, b->stream),
               "resident batch launch");
        }
    }
    // wide instances: lockstep steps, one multi-state launch per step
    if (!b->plan_valid) {
        qsim_status s = build_tiled_plan(b, upload_table);
        if (s != QSIM_OK) return s;
    }
    for (int i = 0; i < b->count; i++) {
        if (b->resident[i]) continue;
        qsim_status s = reset_async(b->inst[i], b->h_init);
        if (s != QSIM_OK) return bfail(b, s, b->inst[i]->err);
    }
    const int threads = b->dtype == QSIM_C64 && b->inst[0]->cfg.fusion == 2 ? 512 : 256;
    for (const auto &st : b->steps) {
        if (st.count)
            CK(qsim::launch_tile_pass_multi(b->dtype, threads, st.kmax, b->d_descs + st.first, st.count,
                                            st.ctas, st.max_m, b->stream),
               "multi-state tile pass launch");
        for (const auto &rg : st.reg)
            CK(qsim::launch_rot_pass_multi(b->d_descs + rg.first, rg.count, rg.ctas, rg.m, rg.dense, b->stream),
               "multi-state register pass launch");
        for (const auto &ev : st.events) {
            qsim_ctx *ic = b->inst[ev.first];
            qsim_status s = launch_measure(ic, (int)ev.second.q, ev.second.flags,
                                           ev.second.ev == qsim::EV_RESET, ic->seed);
            if (s != QSIM_OK) return bfail(b, s, ic->err);
        }
    }
    return QSIM_OK;
}

}  // namespace

extern "C" {

qsim_status qsim_batch_run(qsim_batch *b) {
    if (!b) return fail(nullptr, QSIM_E_INVAL, "null batch");
    qsim_ctx *c = b->aux;
    if (b->graph_exec) {  // replay: one launch for every instance's whole circuit
        CK(cudaGraphLaunch(b->graph_exec, b->stream), "batch graph launch");
        for (int i = 0; i < b->count; i++) b->inst[i]->ordinal = b->inst[i]->log_n = b->meas_after[i];
        return QSIM_OK;
    }
    if (b->eager_runs > 0) {  // capture the run (every allocation was made by the eager one)
        cudaGraph_t g = nullptr;
        if (cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
            qsim_status s = enqueue_run(b, false);
            cudaError_t e = cudaStreamEndCapture(b->stream, &g);
            cudaGraphExec_t ge = nullptr;
            if (s == QSIM_OK && e == cudaSuccess && g &&
                cudaGraphInstantiate(&ge, g, 0) == cudaSuccess) {
                b->graph = g;
                b->graph_exec = ge;
                CK(cudaGraphLaunch(b->graph_exec, b->stream), "batch graph launch");
                return QSIM_OK;
            }
            if (g) cudaGraphDestroy(g);
            cudaGetLastError();
            if (s != QSIM_OK) return s;
        } else {
            cudaGetLastError();
        }
    }
    qsim_status s = enqueue_run(b, true);
    if (s != QSIM_OK) return s;
    b->eager_runs++;
    b->meas_after.resize(b->count);
    for (int i = 0; i < b->count; i++) b->meas_after[i] = b->inst[i]->log_n;
    return QSIM_OK;
}

qsim_status qsim_batch_expect(qsim_batch *b, const qsim_pauli_term *terms, const uint64_t *off,
                              double *out) {
    if (!b || !off) return fail(nullptr, QSIM_E_INVAL, "null argument");
    qsim_ctx *c = b->aux;
    const uint64_t total = off[b->count];
    if (total && (!terms || !out)) return bfail(b, QSIM_E_INVAL, "null terms or out");
    for (int i = 0; i < b->count; i++) {
        if (off[i + 1] < off[i]) return bfail(b, QSIM_E_INVAL, "term offsets must not decrease");
        const int n = b->inst[i]->n;
        const uint64_t full = n >= 64 ? ~0ull : ((1ull << n) - 1ull);
        for (uint64_t t = off[i]; t < off[i + 1]; t++)
            if ((terms[t].x_mask | terms[t].z_mask) & ~full)
                return bfail(b, QSIM_E_INVAL, "Pauli term beyond the instance's qubits");
    }
    if (total == 0) return QSIM_OK;
    const size_t tb = total * 3 * sizeof(uint64_t);
    uint64_t *d_terms = (uint64_t *)dalloc(c, tb);
    double *d_out = (double *)dalloc(c, total * sizeof(double));
    std::vector<qsim::ExpectJob> jobs;
    for (int i = 0; i < b->count; i++) {
        if (!b->resident[i] || off[i + 1] == off[i]) continue;
        // one block per run of terms, at most 2^20 amplitude-terms each, so a
        // wide instance's terms spread over several SMs (each term is still
        // summed by one block in the same order)
        const int n = b->inst[i]->n;
        const uint64_t per = std::max<uint64_t>(1, (1ull << 20) >> n);
        for (uint64_t t0 = off[i]; t0 < off[i + 1]; t0 += per) {
            qsim::ExpectJob j;
            j.state = b->inst[i]->state;
            j.terms = d_terms + 3 * t0;
            j.out = d_out + t0;
            j.n_terms = (uint32_t)std::min<uint64_t>(per, off[i + 1] - t0);
            j.n = n;
            jobs.push_back(j);
        }
    }
    qsim::ExpectJob *d_jobs = (qsim::ExpectJob *)dalloc(c, std::max<size_t>(jobs.size(), 1) * sizeof(qsim::ExpectJob));
    qsim_status s = (d_terms && d_out && d_jobs) ? QSIM_OK : bfail(b, QSIM_E_OOM, "expectation buffers");
    if (s == QSIM_OK) s = upload(c, d_terms, terms, tb);
    if (s == QSIM_OK && !jobs.empty()) s = upload(c, d_jobs, jobs.data(), jobs.size() * sizeof(qsim::ExpectJob));
    if (s == QSIM_OK && !jobs.empty()) {
        cudaError_t e = qsim::launch_expect_batch(b->dtype, d_jobs, (int)jobs.size(), b->stream);
        if (e != cudaSuccess) s = cuda_fail(c, e, "batched expectation launch");
    }
    for (int i = 0; s == QSIM_OK && i < b->count; i++) {
        if (b->resident[i] || off[i + 1] == off[i]) continue;
        qsim_ctx *ic = b->inst[i];
        const size_t nt = off[i + 1] - off[i];
        s = ensure_partials(ic, (size_t)qsim::expect_blocks(ic->n) * nt);
        if (s == QSIM_OK) {
            cudaError_t e = qsim::launch_expect(b->dtype, ic->state, ic->n, d_terms + 3 * off[i], nt,
                                                ic->partials, d_out + off[i], b->stream);
            if (e != cudaSuccess) s = cuda_fail(ic, e, "expectation launch");
        }
    }
    if (s == QSIM_OK) {
        cudaError_t e = cudaMemcpyAsync(out, d_out, total * sizeof(double), cudaMemcpyDeviceToHost, b->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
        if (e != cudaSuccess) s = cuda_fail(c, e, "expectation readback");
    }
    dfree(c, d_terms, tb);
    dfree(c, d_out, total * sizeof(double));
    dfree(c, d_jobs, std::max<size_t>(jobs.size(), 1) * sizeof(qsim::ExpectJob));
    return s == QSIM_OK ? QSIM_OK : bfail(b, s, c->err);
}

qsim_status qsim_batch_state(qsim_batch *b, int index, void *dst, size_t bytes, int dst_is_device) {
    if (!b || index < 0 || index >= b->count) return bfail(b, QSIM_E_INVAL, "bad batch index");
    return qsim_state(b->inst[index], dst, bytes, dst_is_device);
}

qsim_status qsim_batch_outcomes(qsim_batch *b, int index, int32_t *outcomes, double *probs, size_t cap,
                                size_t *n_total) {
    if (!b || index < 0 || index >= b->count) return bfail(b, QSIM_E_INVAL, "bad batch index");
    qsim_ctx *ic = b->inst[index];
    qsim_status s = qsim_outcomes(ic, outcomes, probs, cap, n_total);
    if (s != QSIM_OK) return s;
    return sync_read(ic);
}

qsim_status qsim_batch_resident_count(const qsim_batch *b, int *count) {
    if (!b || !count) return QSIM_E_INVAL;
    int k = 0;
    for (int i = 0; i < b->count; i++) k += b->resident[i];
    *count = k;
    return QSIM_OK;
}

}  // extern "C"

// ------------------------------------------------------------------ serving --
// Requests flow: submit (caller thread) -> pending -> compile workers -> ready
// -> scheduler thread admits into an idle slot (stream) when the request's
// device bytes fit the budget -> completion event -> result queue -> poll.
namespace {

struct ServerReq {
    uint64_t id = 0;
    int n = 0;
    std::vector<qsim_gate> gates;
    std::vector<double> mats;
    uint64_t seed = 0;
    double t_submit = 0, t_admit = 0;
    std::vector<Packed> chunks;
    size_t device_bytes = 0;
    uint64_t n_meas = 0;
    bool cancelled = false;  // its result was delivered by qsim_server_cancel; it never runs
};

struct Slot {
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    qsim_ctx *aux = nullptr;  // staging for uploads on this slot's stream
    std::unique_ptr<ServerReq> req;
    qsim_ctx *ctx = nullptr;  // the running request's state, control block, log
    std::vector<DevChunk> prog;
    // read-back (pinned) and the <Z_q> terms / outputs (device)
    MeasCtl *h_ctl = nullptr;
    MeasRec *h_log = nullptr;
    double *h_z = nullptr;
    uint64_t *d_terms = nullptr;
    double *d_z = nullptr;
};

constexpr int kMaxLog = 64;

double steady_now() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

// A request context created without synchronising: state |0...0> and a
// cleared control block are enqueued on `st`; h_ctl is borrowed.
qsim_ctx *ctx_new_async(int n, qsim_dtype dt, cudaStream_t st, const Config &cfg, MeasCtl *h_ctl,
                        const MeasCtl *h_init) {
    auto *c = new qsim_ctx();
    c->n = n;
    c->dtype = dt;
    c->stream = st;
    c->cfg = cfg;
    cudaGetDevice(&c->device);
    c->state_bytes = (size_t)(dt == QSIM_C64 ? 8 : 16) << n;
    c->state = dalloc(c, c->state_bytes);
    c->ctl = (MeasCtl *)dalloc(c, sizeof(MeasCtl));
    c->h_ctl = h_ctl;
    if (!c->state || !c->ctl || qsim::launch_set_basis(dt, c->state, n, 0, st) != cudaSuccess ||
        cudaMemcpyAsync(c->ctl, h_init, sizeof(MeasCtl), cudaMemcpyHostToDevice, st) != cudaSuccess) {
        cudaGetLastError();
        dfree(c, c->state, c->state_bytes);
        dfree(c, c->ctl, sizeof(MeasCtl));
        delete c;
        return nullptr;
    }
    return c;
}

void ctx_free_async(qsim_ctx *c) {
    dfree(c, c->state, c->state_bytes);
    dfree(c, c->ctl, sizeof(MeasCtl));
    dfree(c, c->log, c->log_cap * sizeof(MeasRec));
    dfree(c, c->partials, c->partials_cap * sizeof(double));
    dfree(c, c->tile_ctr, sizeof(unsigned long long));
    for (auto &s : c->staging) {
        cudaEventSynchronize(s.done);
        cudaEventDestroy(s.done);
        cudaFreeHost(s.host);
    }
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    delete c;  // h_ctl is borrowed from the slot
}

}  // namespace

struct qsim_server {
    qsim_dtype dtype = QSIM_C64;
    Config cfg;
    int device = 0;
    double t0 = 0;
    size_t budget = 0, in_use = 0;
    std::vector<Slot> slots;
    MeasCtl *h_init = nullptr;
    std::mutex mu;
    std::condition_variable cv_work, cv_sched;
    std::deque<std::unique_ptr<ServerReq>> pending;               // to compile
    std::vector<std::unique_ptr<ServerReq>> ready;                // compiled, by id - first_ready_id
    std::vector<ServerReq *> compiling;                           // taken by a compile worker
    uint64_t next_id = 1, next_admit = 1;
    std::vector<qsim_result> results;
    std::atomic<uint64_t> submitted{0}, admitted{0}, completed{0}, running{0}, cancelled{0};
    std::vector<std::thread> workers;
    std::thread sched;
    std::atomic<bool> stop{false};
    std::string err;
};

namespace {

void server_compile_loop(qsim_server *s) {
    for (;;) {
        std::unique_ptr<ServerReq> r;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            s->cv_work.wait(lk, [&] { return s->stop.load() || !s->pending.empty(); });
            if (s->stop.load()) return;
            r = std::move(s->pending.front());
            s->pending.pop_front();
            if (!r->cancelled) s->compiling.push_back(r.get());
        }
        if (r->cancelled) {  // nothing to compile: the scheduler drops it in its turn
            std::vector<qsim_gate>().swap(r->gates);
            std::vector<double>().swap(r->mats);
            std::lock_guard<std::mutex> lk(s->mu);
            const uint64_t idx = r->id - s->next_admit;
            if (s->ready.size() <= idx) s->ready.resize(idx + 1);
            s->ready[idx] = std::move(r);
            s->cv_sched.notify_all();
            continue;
        }
        Config c = s->cfg;
        if (r->n <= qsim::max_resident_bits(s->dtype)) c.tile_bits = r->n;  // one block per request
        HostProgram hp;
        qsim::compile(r->n, s->dtype, c, r->gates.data(), r->gates.size(), r->mats.data(), r->mats.size(), hp);
        Packed pk;
        pack(hp, s->dtype, s->cfg.threads == 0, pk);
        r->n_meas = pk.measurements;
        r->device_bytes = ((size_t)(s->dtype == QSIM_C64 ? 8 : 16) << r->n) + pk.ops.size() * sizeof(DevOp) +
                          pk.mats.size() + (size_t)std::max<uint64_t>(r->n_meas, 1024) * sizeof(MeasRec) +
                          (size_t)qsim::expect_blocks(r->n) * 32 * sizeof(double) + 4096;
        r->chunks.push_back(std::move(pk));
        std::vector<qsim_gate>().swap(r->gates);  // the compiled program replaces the records
        std::vector<double>().swap(r->mats);
        {
            std::lock_guard<std::mutex> lk(s->mu);
            s->compiling.erase(std::find(s->compiling.begin(), s->compiling.end(), r.get()));
            const uint64_t idx = r->id - s->next_admit;  // ready[k] holds id next_admit + k
            if (s->ready.size() <= idx) s->ready.resize(idx + 1);
            s->ready[idx] = std::move(r);
        }
        s->cv_sched.notify_all();
    }
}

void server_finish(qsim_server *s, Slot &sl) {
    ServerReq &r = *sl.req;
    qsim_result res;
    std::memset(&res, 0, sizeof(res));
    res.id = r.id;
    res.n_qubits = r.n;
    res.n_meas = (int32_t)r.n_meas;
    res.status = sl.h_ctl->status;
    res.success = sl.h_ctl->success;
    const int nl = (int)std::min<uint64_t>(r.n_meas, kMaxLog);
    for (int i = 0; i < nl; i++)
        if (sl.h_log[i].outcome == 1) res.outcomes |= 1ull << i;
    const int nz = std::min(r.n, 32);
    for (int q = 0; q < nz; q++) res.z[q] = sl.h_z[q];
    res.t_submit = r.t_submit;
    res.t_admit = r.t_admit;
    res.t_done = steady_now() - s->t0;
    for (auto &dc : sl.prog) release_chunk(sl.aux, dc);
    sl.prog.clear();
    ctx_free_async(sl.ctx);
    sl.ctx = nullptr;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->in_use -= r.device_bytes;
        s->results.push_back(res);
    }
    sl.req.reset();
    s->running--;
    s->completed++;
}

// Enqueue a whole request on an idle slot.  Returns false (with an error
// result delivered) if it could not be enqueued.
bool server_admit(qsim_server *s, Slot &sl, std::unique_ptr<ServerReq> r) {
    r->t_admit = steady_now() - s->t0;
    Config c = s->cfg;
    if (r->n <= qsim::max_resident_bits(s->dtype)) c.tile_bits = r->n;
    qsim_ctx *ctx = ctx_new_async(r->n, s->dtype, sl.stream, c, sl.h_ctl, s->h_init);
    qsim_status st = ctx ? QSIM_OK : QSIM_E_OOM;
    if (ctx) ctx->seed = r->seed;
    for (auto &pk : r->chunks) {
        if (st != QSIM_OK) break;
        DevChunk dc;
        st = upload_chunk(sl.aux, pk, dc);
        sl.prog.push_back(std::move(dc));
    }
    for (auto &dc : sl.prog) {
        if (st != QSIM_OK) break;
        st = launch_chunk(ctx, dc);
    }
    const int nz = std::min(r->n, 32);
    if (st == QSIM_OK) st = ensure_partials(ctx, (size_t)qsim::expect_blocks(r->n) * nz);
    if (st == QSIM_OK && qsim::launch_expect(s->dtype, ctx->state, r->n, sl.d_terms, nz, ctx->partials,
                                             sl.d_z, sl.stream) != cudaSuccess)
        st = QSIM_E_CUDA;
    if (st == QSIM_OK) {
        const int nl = (int)std::min<uint64_t>(r->n_meas, kMaxLog);
        cudaError_t e = cudaMemcpyAsync(sl.h_ctl, ctx->ctl, sizeof(MeasCtl), cudaMemcpyDeviceToHost, sl.stream);
        if (e == cudaSuccess && nl)
            e = cudaMemcpyAsync(sl.h_log, ctx->log, nl * sizeof(MeasRec), cudaMemcpyDeviceToHost, sl.stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(sl.h_z, sl.d_z, nz * sizeof(double), cudaMemcpyDeviceToHost, sl.stream);
        if (e == cudaSuccess) e = cudaEventRecord(sl.done, sl.stream);
        if (e != cudaSuccess) st = QSIM_E_CUDA;
    }
    for (auto &pk : r->chunks) pk = Packed();  // host image no longer needed
    if (st != QSIM_OK) {
        cudaGetLastError();
        cudaStreamSynchronize(sl.stream);
        for (auto &dc : sl.prog) release_chunk(sl.aux, dc);
        sl.prog.clear();
        if (ctx) ctx_free_async(ctx);
        qsim_result res;
        std::memset(&res, 0, sizeof(res));
        res.id = r->id;
        res.n_qubits = r->n;
        res.status = st;
        res.t_submit = r->t_submit;
        res.t_admit = r->t_admit;
        res.t_done = steady_now() - s->t0;
        std::lock_guard<std::mutex> lk(s->mu);
        s->in_use -= r->device_bytes;
        s->results.push_back(res);
        s->completed++;
        return false;
    }
    sl.ctx = ctx;
    sl.req = std::move(r);
    s->running++;
    s->admitted++;
    return true;
}

void server_sched_loop(qsim_server *s) {
    cudaSetDevice(s->device);
    while (!s->stop.load()) {
        bool progress = false;
        for (auto &sl : s->slots)
            if (sl.req && cudaEventQuery(sl.done) == cudaSuccess) {
                server_finish(s, sl);
                progress = true;
            }
        cudaGetLastError();  // cudaErrorNotReady from the queries
        for (auto &sl : s->slots) {
            if (sl.req) continue;
            std::unique_ptr<ServerReq> r;
            {
                std::lock_guard<std::mutex> lk(s->mu);
                if (s->ready.empty() || !s->ready.front()) break;  // strict arrival order
                if (s->ready.front()->cancelled) {  // its result is out already
                    s->ready.erase(s->ready.begin());
                    s->next_admit++;
                    progress = true;
                    continue;
                }
                const size_t need = s->ready.front()->device_bytes;
                const bool alone = s->running.load() == 0;
                if (need > s->budget - s->in_use && !alone) break;  // wait for memory to free up
                r = std::move(s->ready.front());
                s->ready.erase(s->ready.begin());
                s->next_admit++;
                s->in_use += r->device_bytes;
            }
            server_admit(s, sl, std::move(r));
            progress = true;
        }
        if (!progress) {
            std::unique_lock<std::mutex> lk(s->mu);
            s->cv_sched.wait_for(lk, std::chrono::microseconds(50));
        }
    }
}

}  // namespace

extern "C" {

qsim_status qsim_server_destroy(qsim_server *s) {
    if (!s) return QSIM_OK;
    s->stop = true;
    s->cv_work.notify_all();
    s->cv_sched.notify_all();
    for (auto &t : s->workers)
        if (t.joinable()) t.join();
    if (s->sched.joinable()) s->sched.join();
    cudaSetDevice(s->device);
    for (auto &sl : s->slots) {
        if (sl.stream) cudaStreamSynchronize(sl.stream);
        if (sl.req) {
            for (auto &dc : sl.prog) release_chunk(sl.aux, dc);
            if (sl.ctx) ctx_free_async(sl.ctx);
        }
        if (sl.aux) {
            dfree(sl.aux, sl.d_terms, 32 * 3 * sizeof(uint64_t));
            dfree(sl.aux, sl.d_z, 32 * sizeof(double));
            qsim_destroy(sl.aux);
        }
        if (sl.stream) cudaStreamSynchronize(sl.stream);
        if (sl.done) cudaEventDestroy(sl.done);
        if (sl.stream) cudaStreamDestroy(sl.stream);
        if (sl.h_ctl) cudaFreeHost(sl.h_ctl);
        if (sl.h_log) cudaFreeHost(sl.h_log);
        if (sl.h_z) cudaFreeHost(sl.h_z);
    }
    if (s->h_init) cudaFreeHost(s->h_init);
    cudaGetLastError();
    delete s;
    return QSIM_OK;
}

qsim_status qsim_server_create(int slots, size_t mem_budget, qsim_dtype dtype, const qsim_config *cfg,
                               int compile_threads, qsim_server **out) {
    if (!out) return fail(nullptr, QSIM_E_INVAL, "out is NULL");
    *out = nullptr;
    if (slots < 1 || slots > 64) return fail(nullptr, QSIM_E_INVAL, "slots must be in [1, 64]");
    if (dtype != QSIM_C64 && dtype != QSIM_C128) return fail(nullptr, QSIM_E_INVAL, "bad dtype");
    {
        std::string err;
        if (cfg && !check_config(cfg, dtype, 0, err)) return fail(nullptr, QSIM_E_INVAL, err);
    }
    auto s = std::make_unique<qsim_server>();
    s->dtype = dtype;
    s->cfg = qsim::config_from(cfg);
    s->t0 = steady_now();
    if (cudaGetDevice(&s->device) != cudaSuccess) {
        cudaGetLastError();
        return fail(nullptr, QSIM_E_CUDA, "no CUDA device");
    }
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
        cudaGetLastError();
        return fail(nullptr, QSIM_E_CUDA, "cudaMemGetInfo");
    }
    s->budget = mem_budget ? mem_budget : (size_t)(0.8 * (double)free_b);
    if (cudaMallocHost((void **)&s->h_init, sizeof(MeasCtl)) != cudaSuccess) {
        cudaGetLastError();
        return fail(nullptr, QSIM_E_OOM, "pinned memory");
    }
    std::memset(s->h_init, 0, sizeof(MeasCtl));
    s->h_init->success = 1.0;
    // <Z_q> terms for q < 32, shared layout with qsim_pauli_term
    std::vector<uint64_t> zt(32 * 3, 0);
    const double one = 1.0;
    for (int q = 0; q < 32; q++) {
        zt[3 * q + 1] = 1ull << q;
        std::memcpy(&zt[3 * q + 2], &one, sizeof(one));
    }
    s->slots.resize(slots);
    for (auto &sl : s->slots) {
        bool ok = cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) == cudaSuccess &&
                  cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming) == cudaSuccess &&
                  cudaMallocHost((void **)&sl.h_ctl, sizeof(MeasCtl)) == cudaSuccess &&
                  cudaMallocHost((void **)&sl.h_log, kMaxLog * sizeof(MeasRec)) == cudaSuccess &&
                  cudaMallocHost((void **)&sl.h_z, 32 * sizeof(double)) == cudaSuccess;
        if (ok) ok = qsim_create(1, dtype, sl.stream, nullptr, nullptr, nullptr, &sl.aux) == QSIM_OK;
        if (ok) {
            sl.d_terms = (uint64_t *)dalloc(sl.aux, zt.size() * sizeof(uint64_t));
            sl.d_z = (double *)dalloc(sl.aux, 32 * sizeof(double));
            ok = sl.d_terms && sl.d_z && upload(sl.aux, sl.d_terms, zt.data(), zt.size() * sizeof(uint64_t)) == QSIM_OK &&
                 cudaStreamSynchronize(sl.stream) == cudaSuccess;
        }
        if (!ok) {
            cudaGetLastError();
            qsim_server_destroy(s.release());
            return fail(nullptr, QSIM_E_CUDA, "server slot set-up failed");
        }
    }
    int T = compile_threads > 0 ? compile_threads
                                : (int)std::max(1u, std::min(std::thread::hardware_concurrency() / 2, 16u));
    qsim_server *raw = s.get();
    for (int t = 0; t < T; t++) s->workers.emplace_back(server_compile_loop, raw);
    s->sched = std::thread(server_sched_loop, raw);
    *out = s.release();
    return QSIM_OK;
}

double qsim_server_now(const qsim_server *s) { return s ? steady_now() - s->t0 : 0.0; }

qsim_status qsim_server_submit(qsim_server *s, int n, const qsim_gate *g, size_t ng, const double *mats,
                               size_t nm, uint64_t seed, double t_submit, uint64_t *id) {
    if (!s) return fail(nullptr, QSIM_E_INVAL, "null server");
    if (n < 1 || n > 34) return fail(nullptr, QSIM_E_INVAL, "n_qubits must be in [1, 34]");
    if (ng && !g) return fail(nullptr, QSIM_E_INVAL, "gates is NULL");
    std::string err;
    if (!qsim::validate(n, g, ng, mats, nm, err)) return fail(nullptr, QSIM_E_INVAL, err);
    auto r = std::make_unique<ServerReq>();
    r->n = n;
    r->gates.assign(g, g + ng);
    if (mats && nm) r->mats.assign(mats, mats + nm);
    r->seed = seed;
    r->t_submit = t_submit >= 0 ? t_submit : steady_now() - s->t0;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        r->id = s->next_id++;
        if (id) *id = r->id;
        s->pending.push_back(std::move(r));
    }
    s->submitted++;
    s->cv_work.notify_one();
    return QSIM_OK;
}

qsim_status qsim_server_poll(qsim_server *s, qsim_result *out, size_t cap, size_t *n_out) {
    if (!s) return fail(nullptr, QSIM_E_INVAL, "null server");
    std::lock_guard<std::mutex> lk(s->mu);
    const size_t k = std::min(cap, s->results.size());
    if (k) {
        std::memcpy(out, s->results.data(), k * sizeof(qsim_result));
        s->results.erase(s->results.begin(), s->results.begin() + k);
    }
    if (n_out) *n_out = k;
    return QSIM_OK;
}

qsim_status qsim_server_counts(const qsim_server *s, uint64_t *submitted, uint64_t *admitted,
                               uint64_t *completed, uint64_t *pending, uint64_t *running) {
    if (!s) return QSIM_E_INVAL;
    const uint64_t sub = s->submitted.load(), adm = s->admitted.load(), done = s->completed.load();
    if (submitted) *submitted = sub;
    if (admitted) *admitted = adm;
    if (completed) *completed = done;
    if (running) *running = s->running.load();
    const uint64_t can = s->cancelled.load();
    if (pending) *pending = sub >= adm + can ? sub - adm - can : 0;
    return QSIM_OK;
}

qsim_status qsim_server_cancel(qsim_server *s, uint64_t id) {
    if (!s) return fail(nullptr, QSIM_E_INVAL, "null server");
    std::lock_guard<std::mutex> lk(s->mu);
    ServerReq *r = nullptr;
    for (auto &p : s->pending)
        if (p->id == id) r = p.get();
    for (ServerReq *p : s->compiling)
        if (p->id == id) r = p;
    if (!r && id >= s->next_admit && id - s->next_admit < s->ready.size() && s->ready[id - s->next_admit])
        r = s->ready[id - s->next_admit].get();
    if (!r || r->cancelled) return fail(nullptr, QSIM_E_INVAL, "request " + std::to_string(id) + " is not waiting");
    r->cancelled = true;
    qsim_result res;
    std::memset(&res, 0, sizeof(res));
    res.id = r->id;
    res.status = QSIM_E_CANCELED;
    res.n_qubits = r->n;
    res.success = 1.0;
    res.t_submit = r->t_submit;
    res.t_admit = -1.0;
    res.t_done = steady_now() - s->t0;
    s->results.push_back(res);
    s->cancelled++;
    s->completed++;
    return QSIM_OK;
}

}  // extern "C"
