// hj_tc.cu -- tensor-core (tcgen05) tile kernel of the linear-quadratic
// family H = <A x, p> + |B^T p|^2 / 2 (fp32 contexts).
//
// The characteristic field of this family is linear (Sec. 4.1 system with
// dH/dp = A gamma + B B^T p, dH/dx = A^T p), so every RK4 stage of every
// (query, start) pair is a product of one fixed matrix with the pair's
// stage vector.  A CTA owns a tile of 128 pairs, one per TMEM lane (two
// threads per pair split its columns), and evaluates each stage for all of
// them as tensor-core products [128 x K] x [K x N]:
//   forward  Z_s = (gamma_s, p_s)                 -> (k_gamma, k_p, y = B^T p_s)
//            k_gamma = -(A gamma_s + C p_s), k_p = A^T p_s, C = B B^T,
//            running cost L_s = |y|^2 / 2 (Lax and Hopf alike);
//   reverse  (w_gamma, w_p, b y_s)                 -> (r_gamma, r_p)
//            r_gamma = -A^T w_gamma, r_p = A w_p - C w_gamma + b B y_s,
// the vector-Jacobian product of the discrete adjoint of RK4 (the y_s of
// the forward pass are kept in global memory, so no state is recomputed).
// Each pass is one dense product (N = 2 dp + mp or 2 dp columns): a K=16
// MMA costs about the same for N = 64 as for N = 160, so skipping the zero
// blocks of the matrices with narrower products is slower.
// Products are split-precision BF16x3: each fp32 operand x = hi + lo with
// hi = bf16(x), lo = bf16(x - hi), and the product is hi*hi + hi*lo + lo*hi
// accumulated in fp32 in tensor memory (relative error ~2^-16).
//
// Operands sit in shared memory in the no-swizzle K-major layout of 8x8
// bf16 core matrices (128 B each; K-adjacent cores 128 B apart, 8-row groups
// (K/8)*128 B apart); the fixed matrix of the pass is copied in once per
// pass, the stage tile is written by the epilogue threads.  Tensor memory
// holds the accumulator and, as per-thread extra storage, the RK4 state and
// stage sums (forward) or the adjoint state and stage sums (reverse).
//
// Thread 0 issues the MMAs and commits them to an mbarrier; every wait on
// it is bounded and a timeout sets the error word, abandons the tile and
// frees the tensor memory.
#include <cuda_bf16.h>

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <vector>

#include "hj_device.cuh"
#include "hj_kernels.cuh"
#include "hj_tc.h"

namespace hjd {

namespace {

constexpr int TCR = 128;         // pairs (rows) per tile = TMEM lanes
constexpr int TPR = 2;           // threads per row (pair): they take alternate 16-column chunks
constexpr int TCT = TCR * TPR;   // threads per CTA
constexpr uint32_t TM_COLS = 512;
constexpr uint32_t COL_Z = 256;  // forward: z (RK4 state) columns; reverse: lambda
constexpr long long WAIT_LIMIT = 1ll << 22;

__device__ __forceinline__ uint32_t s_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor: K-major, no swizzle, K-adjacent core
// matrices 128 B apart (leading byte offset), 8-row groups `sbo` apart.
__device__ __forceinline__ uint64_t mdesc(uint32_t addr, uint32_t sbo)
{
    return (uint64_t)((addr & 0x3FFFF) >> 4) | ((uint64_t)(128 >> 4) << 16) | ((uint64_t)(sbo >> 4) << 32) |
           (1ull << 46);
}

// Instruction descriptor of kind::f16: bf16 A and B (K-major), f32 D, M x N.
__device__ __forceinline__ uint32_t idesc_bf16(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t dtm, uint64_t a, uint64_t b, uint32_t id, uint32_t acc)
{
    asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                 "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(dtm),
                 "l"(a), "l"(b), "r"(id), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint32_t mbar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
                 : "memory");
}

// Bounded wait for the mbarrier phase of the given parity; false on timeout.
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity)
{
    uint32_t done = 0;
    for (long long it = 0; it < WAIT_LIMIT; ++it) {
        asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                     "selp.u32 %0, 1, 0, p;\n}"
                     : "=r"(done)
                     : "r"(mbar), "r"(parity)
                     : "memory");
        if (done) return true;
    }
    return false;
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tm_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void tm_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// 16 consecutive TMEM columns of this thread's lane.
__device__ __forceinline__ void tm_ld16(uint32_t ta, float *v)
{
    uint32_t r[16];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
                 "[%16];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                   "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                   "=r"(r[15])
                 : "r"(ta)
                 : "memory");
#pragma unroll
    for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}
__device__ __forceinline__ void tm_st16(uint32_t ta, const float *v)
{
    asm volatile("tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                 "%16};" ::"r"(ta),
                 "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])),
                 "r"(__float_as_uint(v[3])), "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])),
                 "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7])), "r"(__float_as_uint(v[8])),
                 "r"(__float_as_uint(v[9])), "r"(__float_as_uint(v[10])), "r"(__float_as_uint(v[11])),
                 "r"(__float_as_uint(v[12])), "r"(__float_as_uint(v[13])), "r"(__float_as_uint(v[14])),
                 "r"(__float_as_uint(v[15]))
                 : "memory");
}

// Byte offset of element (r, k) of a K-major core-matrix tile with kc columns.
__device__ __forceinline__ uint32_t tile_off(int r, int k, int kc)
{
    return (uint32_t)((r >> 3) * (kc >> 3) * 128 + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2);
}

// hi/lo bf16 split of 8 floats, packed as two 16-byte core-matrix rows.
__device__ __forceinline__ void split8(const float *f, uint4 &hi, uint4 &lo)
{
    uint32_t h[4], l[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const __nv_bfloat162 hb = __floats2bfloat162_rn(f[2 * j], f[2 * j + 1]);
        const float r0 = f[2 * j] - __low2float(hb), r1 = f[2 * j + 1] - __high2float(hb);
        const __nv_bfloat162 lb = __floats2bfloat162_rn(r0, r1);
        h[j] = *(const uint32_t *)&hb;
        l[j] = *(const uint32_t *)&lb;
    }
    hi = make_uint4(h[0], h[1], h[2], h[3]);
    lo = make_uint4(l[0], l[1], l[2], l[3]);
}

// Row `r`, columns c..c+15 of the stage tile (hi and lo copies).
__device__ __forceinline__ void put16(unsigned char *zh, unsigned char *zl, int r, int c, int kc, const float *v)
{
    uint4 h, l;
    split8(v, h, l);
    *(uint4 *)(zh + tile_off(r, c, kc)) = h;
    *(uint4 *)(zl + tile_off(r, c, kc)) = l;
    split8(v + 8, h, l);
    *(uint4 *)(zh + tile_off(r, c + 8, kc)) = h;
    *(uint4 *)(zl + tile_off(r, c + 8, kc)) = l;
}

struct Tile {
    // shared memory
    unsigned char *wh, *wl, *zh, *zl;
    uint32_t mbar;
    uint32_t phase;
    uint32_t tm;    // TMEM base (lane 0, column 0)
    uint32_t lane;  // this warp's lane quarter, in TMEM address form
    int row;        // tile row (pair) of this thread
    int half;       // which half of the row's column chunks this thread handles
    bool abort;
};

__device__ __forceinline__ uint32_t ta(const Tile &T, uint32_t col) { return T.tm + T.lane + col; }

// Copy a pass's fixed matrices (core-matrix layout, hi and lo) into shared memory.
__device__ __forceinline__ void load_matrix(const Tile &T, const uint4 *hi, const uint4 *lo, int bytes)
{
    const int n = bytes >> 4;
    for (int i = threadIdx.x; i < n; i += TCT) {
        ((uint4 *)T.wh)[i] = __ldg(hi + i);
        ((uint4 *)T.wl)[i] = __ldg(lo + i);
    }
}

// One stage: waits for every thread's tile writes, issues the pass's
// products (each three BF16x3 terms of K/16 MMAs) and waits for them.
// Returns false (abort, taken by every thread alike) on a timeout.
__device__ __forceinline__ bool stage_mma(Tile &T, const LqTcProd *pr, int kz)
{
    fence_proxy();
    tm_wait_st();
    fence_before();
    __syncthreads();
    if (threadIdx.x == 0) {
        fence_after();
        const uint32_t zh = s_addr(T.zh), zl = s_addr(T.zl), wh = s_addr(T.wh), wl = s_addr(T.wl);
        const uint32_t sbo_z = (uint32_t)(kz >> 3) * 128;
        for (int i = 0; i < 1; ++i) {
            const LqTcProd P = pr[i];
            const uint32_t id = idesc_bf16(TCR, P.N), sbo_w = (uint32_t)(P.kw >> 3) * 128;
            const uint32_t ao = (uint32_t)(P.acol >> 3) * 128;
            for (int term = 0; term < 3; ++term) {
                const uint32_t a = ((term == 2) ? zl : zh) + ao, b = ((term == 1) ? wl : wh) + P.boff;
                for (int kk = 0; kk < P.K / 16; ++kk)
                    mma_bf16(T.tm + P.dcol, mdesc(a + kk * 256, sbo_z), mdesc(b + kk * 256, sbo_w), id,
                             (term | kk) ? 1u : 0u);
            }
        }
        mma_commit(T.mbar);
    }
    const bool ok = mbar_wait(T.mbar, T.phase);
    T.phase ^= 1;
    if (__syncthreads_or(ok ? 0 : 1)) {
        T.abort = true;
        return false;
    }
    fence_after();
    return true;
}

}  // namespace

// ---------------------------------------------------------------------------
// Per-row inputs and outputs of a tile evaluation.
// ---------------------------------------------------------------------------
struct RowIO {
    int N;       // RK4 steps (0: masked row)
    float h;     // t / N
    float F;     // out: functional
    float resid; // out: certificate residual at (gamma(0), p(0))
};

// F at the points PT (and its gradient into G when `grad`) for the 128 rows
// of the tile.  X, PT, G are this CTA's component-major scratch (entry
// [k * 128 + row]); ybuf: this CTA's stage outputs y (grad only).  The two
// threads of a row take alternate 16-column chunks; per-row sums are
// combined through `red` (shared, [3][TPR][128]).
__device__ bool tile_eval(Tile &T, const LqTcArgs &a, bool grad, const float *X, const float *PT, float *G,
                          float *ybuf, RowIO &io, int nmax, float *red)
{
    const int r = T.row, c0 = 16 * T.half, d = a.d, dp = a.dp, mp = a.mp, kz = a.KZ;
    const int d2 = 2 * dp;
    const bool live_row = io.N > 0;
    const float h = io.h;
    // ---- forward pass --------------------------------------------------------
    __syncthreads();  // the previous pass's products have completed; W may be overwritten
    load_matrix(T, a.wf_hi, a.wf_lo, (int)a.w_bytes);
    for (int c = c0; c < d2; c += 16 * TPR) {
        float z[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            const int k = c + j;
            float val = 0.f;
            if (k < dp) { if (k < d) val = X[k * TCR + r]; }
            else if (k - dp < d) val = PT[(k - dp) * TCR + r];
            z[j] = val;
        }
        tm_st16(ta(T, COL_Z + c), z);
        put16(T.zh, T.zl, r, c, kz, z);
    }
    float Q = 0.f, Qc = 0.f, La = 0.f;  // this thread's share of the quadrature
    for (int n = 0; n < nmax; ++n) {
        const bool live = live_row && n < io.N;
        for (int s = 1; s <= 4; ++s) {
            if (!stage_mma(T, a.fwd, kz)) return false;
            const float cn = (s == 3) ? h : 0.5f * h, h6 = h / 6.f;
            for (int c = c0; c < d2; c += 16 * TPR) {
                float k[16], z[16], ks[16], zn[16];
                tm_ld16(ta(T, c), k);
                tm_ld16(ta(T, COL_Z + c), z);
                if (s > 1) tm_ld16(ta(T, COL_Z + d2 + c), ks);
                tm_wait_ld();
                if (s < 4) {
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        ks[j] = (s == 1) ? k[j] : fmaf(2.f, k[j], ks[j]);
                        zn[j] = fmaf(cn, k[j], z[j]);
                    }
                    tm_st16(ta(T, COL_Z + d2 + c), ks);
                } else {
#pragma unroll
                    for (int j = 0; j < 16; ++j) zn[j] = live ? fmaf(h6, ks[j] + k[j], z[j]) : z[j];
                    tm_st16(ta(T, COL_Z + c), zn);  // .sync.aligned: every lane stores
                }
                put16(T.zh, T.zl, r, c, kz, zn);
            }
            float Ls = 0.f;
            for (int c = c0; c < mp; c += 16 * TPR) {
                float y[16];
                tm_ld16(ta(T, d2 + c), y);
                tm_wait_ld();
#pragma unroll
                for (int j = 0; j < 16; ++j) Ls = fmaf(y[j], y[j], Ls);
                if (grad) {
                    float *yb = ybuf + ((size_t)(n * 4 + s - 1) * mp + c) * TCR + r;
#pragma unroll
                    for (int j = 0; j < 16; ++j) yb[(size_t)j * TCR] = live ? y[j] : 0.f;
                }
            }
            Ls *= 0.5f;
            La = (s == 1) ? Ls : (s == 4 ? La + Ls : fmaf(2.f, Ls, La));
        }
        if (live) {
            // Kahan-compensated quadrature sum
            const float dQ = h / 6.f * La;
            const float yk = dQ - Qc, sk = Q + yk;
            Qc = (sk - Q) - yk;
            Q = sk;
        }
    }
    // ---- terminal term, adjoint seed, certificate residual ------------------
    float term = 0.f, num = 0.f, den = 0.f;
    for (int c = c0; c < dp; c += 16 * TPR) {
        float gm[16], pm[16], lg[16], lp[16];
        tm_ld16(ta(T, COL_Z + c), gm);
        tm_ld16(ta(T, COL_Z + dp + c), pm);
        tm_wait_ld();
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            const int i = c + j;  // < dp <= DPAD: parameter vectors are zero padded
            lg[j] = lp[j] = 0.f;
            if (a.principle == HJ_LAX) {
                const float gr = (a.g_kind == HJ_G_QUAD_SHIFT) ? gm[j] - __ldg(a.ga + i) : gm[j] * __ldg(a.gis2 + i);
                term = fmaf(0.5f * gr, (a.g_kind == HJ_G_QUAD_SHIFT) ? gr : gm[j], term);
                lg[j] = gr;
                const float df = pm[j] - gr;
                num = fmaf(df, df, num);
                den = fmaf(pm[j], pm[j], den);
            } else {
                float gr, val;
                if (a.g_kind == HJ_G_QUAD_SHIFT) {
                    const float av = __ldg(a.ga + i);
                    gr = pm[j] + av;
                    val = pm[j] * fmaf(0.5f, pm[j], av);
                } else {
                    gr = __ldg(a.gs2 + i) * pm[j];
                    val = 0.5f * gr * pm[j];
                }
                const float xv = (i < d) ? X[i * TCR + r] : 0.f, vv = (i < d) ? PT[i * TCR + r] : 0.f;
                term += val - xv * vv;
                lp[j] = gr;
                const float df = gm[j] - gr;
                num = fmaf(df, df, num);
                den = fmaf(gm[j], gm[j], den);
            }
        }
        if (grad) {
            tm_st16(ta(T, COL_Z + c), lg);       // lambda_gamma
            tm_st16(ta(T, COL_Z + dp + c), lp);  // lambda_p
        }
    }
    // combine the row's threads' sums
    red[(0 * TPR + T.half) * TCR + r] = term + Q;
    red[(1 * TPR + T.half) * TCR + r] = num;
    red[(2 * TPR + T.half) * TCR + r] = den;
    __syncthreads();
    {
        float F = 0.f, nm = 0.f, dn = 0.f;
#pragma unroll
        for (int k = 0; k < TPR; ++k) {
            F += red[(0 * TPR + k) * TCR + r];
            nm += red[(1 * TPR + k) * TCR + r];
            dn += red[(2 * TPR + k) * TCR + r];
        }
        io.F = live_row ? F : __int_as_float(0x7fc00000);
        io.resid = sqrtf(nm) / (1.f + sqrtf(dn));
    }
    if (!grad) {
        __syncthreads();  // red may be reused
        return true;
    }

    // ---- reverse pass (discrete adjoint of RK4) ------------------------------
    // tensor memory: [0, 2dp) the product a_s, [COL_Z, +2dp) lambda,
    // [COL_Z + 2dp, +2dp) the running sum of a_s over the step's stages
    fence_before();
    __syncthreads();  // every forward product has completed: W may be replaced
    load_matrix(T, a.wv_hi, a.wv_lo, (int)a.w_bytes);
    tm_wait_st();
    // input of stage (n, s): w = c1 lambda + c2 a_prev on the state columns,
    // b y_s on the y columns; masked rows feed zeros.  The y of the next
    // input are loaded before the current stage's product is awaited, so the
    // global-memory latency overlaps the tensor-core work.
    // (the first y chunk of this thread is prefetched; a second one, when
    // mp > 32, is read when it is written)
    float ypre[16];
    int y_n = 0, y_s = 0;
    float y_b = 0.f;
    auto read_y = [&](int n, int s, float b, int c, float *y) {
        const bool live = live_row && n >= 0 && n < io.N;
        const float *yb = ybuf + ((size_t)(n * 4 + s - 1) * mp + c) * TCR + r;
#pragma unroll
        for (int j = 0; j < 16; ++j) y[j] = live ? b * yb[(size_t)j * TCR] : 0.f;
    };
    auto load_y = [&](int n, int s, float b) {
        y_n = n;
        y_s = s;
        y_b = b;
        if (c0 < mp) read_y(n, s, b, c0, ypre);
    };
    auto put_y = [&]() {
        if (c0 < mp) put16(T.zh, T.zl, r, d2 + c0, kz, ypre);
        for (int c = c0 + 16 * TPR; c < mp; c += 16 * TPR) {
            float y[16];
            read_y(y_n, y_s, y_b, c, y);
            put16(T.zh, T.zl, r, d2 + c, kz, y);
        }
    };
    {
        const int n = nmax - 1;
        const bool live = live_row && n < io.N;
        for (int c = c0; c < d2; c += 16 * TPR) {
            float lm[16], w[16];
            tm_ld16(ta(T, COL_Z + c), lm);
            tm_wait_ld();
#pragma unroll
            for (int j = 0; j < 16; ++j) w[j] = live ? h / 6.f * lm[j] : 0.f;
            put16(T.zh, T.zl, r, c, kz, w);
        }
        load_y(n, 4, h / 6.f);
        put_y();
    }
    for (int n = nmax - 1; n >= 0; --n) {
        for (int s = 4; s >= 1; --s) {
            // next input: (n, s-1), or (n-1, 4) after the step's last stage
            const int nn = (s > 1) ? n : n - 1;
            const int sn = (s > 1) ? s - 1 : 4;
            if (nn >= 0) load_y(nn, sn, (sn == 3 || sn == 2) ? h / 3.f : h / 6.f);
            if (!stage_mma(T, a.rev, kz)) return false;
            const bool live_n = live_row && nn >= 0 && nn < io.N;
            const float c1 = (sn == 3 || sn == 2) ? h / 3.f : h / 6.f;
            const float c2 = (sn == 3) ? h : 0.5f * h;
            for (int c = c0; c < d2; c += 16 * TPR) {
                float av[16], lm[16], as[16], w[16];
                tm_ld16(ta(T, c), av);
                tm_ld16(ta(T, COL_Z + c), lm);
                if (s < 4) tm_ld16(ta(T, COL_Z + d2 + c), as);
                tm_wait_ld();
                if (s > 1) {
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        as[j] = (s == 4) ? av[j] : as[j] + av[j];
                        w[j] = live_n ? fmaf(c1, lm[j], c2 * av[j]) : 0.f;
                    }
                    tm_st16(ta(T, COL_Z + d2 + c), as);
                } else {
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        lm[j] += as[j] + av[j];
                        w[j] = live_n ? h / 6.f * lm[j] : 0.f;
                    }
                    tm_st16(ta(T, COL_Z + c), lm);
                }
                if (nn >= 0) put16(T.zh, T.zl, r, c, kz, w);
            }
            if (nn >= 0) put_y();
        }
    }
    // dF/dv = lambda_p at tau = 0 (minus x for Hopf)
    for (int c = c0; c < dp; c += 16 * TPR) {
        float lp[16];
        tm_ld16(ta(T, COL_Z + dp + c), lp);
        tm_wait_ld();
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            const int i = c + j;
            if (i < d) G[i * TCR + r] = (a.principle == HJ_HOPF) ? lp[j] - X[i * TCR + r] : lp[j];
        }
    }
    __syncthreads();  // G complete for the row's first thread
    return true;
}

// ---------------------------------------------------------------------------
// The kernel: rows mode (functional, gradient) or the persistent descent.
// Threads t, t + 128, ... share row t % 128; per-row bookkeeping (inputs,
// descent, outputs) is done by the first of them.
// ---------------------------------------------------------------------------
template <int MODE>
__global__ void __launch_bounds__(TCT, 1) k_lq_tc(LqTcArgs a)
{
    extern __shared__ __align__(1024) unsigned char dsm[];
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tslot;
    __shared__ int s_nmax;
    __shared__ float s_red[3 * TPR * TCR];
    const int tid = threadIdx.x, warp = tid >> 5;
    Tile T;
    T.wh = dsm;
    T.wl = dsm + a.w_bytes;
    T.zh = dsm + 2 * a.w_bytes;
    T.zl = dsm + 2 * a.w_bytes + a.z_bytes;
    T.mbar = s_addr(&mbar);
    T.phase = 0;
    T.lane = (uint32_t)((warp & 3) * 32) << 16;
    T.row = tid & (TCR - 1);
    T.half = tid / TCR;
    T.abort = false;
    const int r = T.row;
    const bool lead = T.half == 0;
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(T.mbar));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(s_addr(&tslot)),
                     "r"(TM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    fence_before();
    __syncthreads();
    fence_after();
    T.tm = tslot;

    float *X = a.vec + (size_t)blockIdx.x * a.vec_slot;
    float *V = X + (size_t)a.dp * TCR, *P1 = V + (size_t)a.dp * TCR, *P2 = P1 + (size_t)a.dp * TCR;
    float *PT = P2 + (size_t)a.dp * TCR, *G = PT + (size_t)a.dp * TCR;
    float *ybuf = a.ybuf + (size_t)blockIdx.x * a.ybuf_slot;
    const int d = a.d;
    unsigned long long n_it = 0, n_g = 0, n_rk = 0, n_adj = 0, n_pairs = 0, n_sumN = 0, n_cert = 0;

    long long n_rows, begin = 0;
    if (MODE == LQ_DESC) {
        n_rows = a.D.wl_count[a.D.problem];
        begin = a.D.seg_begin[a.D.problem];
    } else {
        n_rows = a.n;
    }
    for (long long tile = blockIdx.x; tile * TCR < n_rows; tile += gridDim.x) {
        const long long j = tile * TCR + r;
        bool valid = j < n_rows;
        long long pid = -1, q = -1;
        if (valid) {
            if (MODE == LQ_DESC) {
                pid = a.D.wl[begin + j];
                q = a.D.pair_q[pid];
            } else {
                q = pid = j;
                if (a.pidx && a.pidx[j] != a.pfilter) valid = false;
            }
        }
        int N = 0;
        float t = 0.f;
        if (valid) {
            N = a.nsteps ? a.nsteps[q] : a.n_default;
            t = a.t[q];
        }
        const bool n_ok = (N >= 1 && N <= MAX_N);
        RowIO io;
        io.N = (valid && n_ok) ? N : 0;
        io.h = (valid && n_ok) ? t / (float)N : 0.f;
        // inputs into the component-major scratch
        if (lead)
            for (int k = 0; k < d; ++k) {
                X[k * TCR + r] = valid ? a.x[q * a.ld + k] : 0.f;
                float v0 = 0.f;
                if (valid) {
                    if (MODE == LQ_DESC)
                        v0 = start_component<float>(a.D.S.seed, a.D.q_begin + q, a.D.pair_slot[pid],
                                                    a.D.pair_round[pid], k, a.D.S.guess_dist);
                    else
                        v0 = a.v[pid * a.ld + k];
                }
                V[k * TCR + r] = v0;
                PT[k * TCR + r] = v0;
            }
        if (tid == 0) s_nmax = 0;
        __syncthreads();
        if (lead && io.N > 0) atomicMax(&s_nmax, io.N);
        __syncthreads();
        const int nmax = s_nmax;

        if (MODE != LQ_DESC) {
            if (nmax > 0 && !tile_eval(T, a, MODE == LQ_ROWS_GRAD, X, PT, G, ybuf, io, nmax, s_red)) break;
            if (valid && lead) {
                const float nanv = __int_as_float(0x7fc00000);
                if (a.F) a.F[pid] = (io.N > 0) ? io.F : nanv;
                if (MODE == LQ_ROWS_GRAD)
                    for (int k = 0; k < d; ++k) a.grad[pid * a.ld + k] = (io.N > 0) ? G[k * TCR + r] : nanv;
            }
            continue;
        }

        // ---- descent: gradient (DESC_GD) or conjugate-gradient (DESC_CG) steps ----
        const SolverDev &S = a.D.S;
        int it = 0, phase = 0, bad = 0;
        bool active = lead && valid && S.max_iters > 0, conv = false;
        if (valid && !n_ok) { active = false; bad = 1; }
        float sig = 0.f, dn = 0.f;
        if (lead)
            for (int k = 0; k < d; ++k) {
                P1[k * TCR + r] = 0.f;                                              // previous gradient
                P2[k * TCR + r] = (a.mode_desc == DESC_GD) ? (float)S.step : 0.f;  // alpha (GD) / direction (CG)
            }
        bool aborted = false;
        while (__syncthreads_or(active ? 1 : 0)) {
            if (lead) {
                if (a.mode_desc == DESC_CG && phase == 1)
                    for (int k = 0; k < d; ++k) PT[k * TCR + r] = fmaf(sig, P2[k * TCR + r], V[k * TCR + r]);
                else
                    for (int k = 0; k < d; ++k) PT[k * TCR + r] = V[k * TCR + r];
            }
            if (!tile_eval(T, a, true, X, PT, G, ybuf, io, nmax, s_red)) { aborted = true; break; }
            if (!active) continue;
            n_g++;
            n_rk += io.N;
            n_adj += io.N;
            bool stop = false;
            if (a.mode_desc == DESC_GD) {
                float big = 0.f;
                bool fin = true;
                for (int k = 0; k < d; ++k) {
                    const float gk = G[k * TCR + r];
                    float al = P2[k * TCR + r];
                    if (S.adapt) {
                        const float prod = gk * P1[k * TCR + r];
                        if (prod < 0.f) al *= (float)S.shrink;
                        else if (prod > 0.f) al = fminf(al * (float)S.grow, (float)S.step_max);
                    }
                    const float st = al * gk;
                    fin = fin && isfinite(st);
                    V[k * TCR + r] -= st;
                    big = fmaxf(big, fabsf(st));
                    P1[k * TCR + r] = gk;
                    P2[k * TCR + r] = al;
                }
                ++it;
                if (!fin) { bad = 1; stop = true; }
                if (S.halving_period > 0 && it % S.halving_period == 0)
                    for (int k = 0; k < d; ++k) P2[k * TCR + r] *= 0.5f;
                if (!stop && big < (float)S.eps) conv = stop = true;
            } else if (phase == 0) {
                if (it == 0) {
                    for (int k = 0; k < d; ++k) P2[k * TCR + r] = -G[k * TCR + r];
                } else {
                    float gg = 0.f, gy = 0.f;
                    for (int k = 0; k < d; ++k) {
                        const float gk = G[k * TCR + r], pk = P1[k * TCR + r];
                        gg = fmaf(pk, pk, gg);
                        gy = fmaf(gk, gk - pk, gy);
                    }
                    const float beta = (gg > 0.f) ? fmaxf(0.f, gy / gg) : 0.f;
                    float gd = 0.f;
                    for (int k = 0; k < d; ++k) {
                        const float dk = fmaf(beta, P2[k * TCR + r], -G[k * TCR + r]);
                        P2[k * TCR + r] = dk;
                        gd = fmaf(G[k * TCR + r], dk, gd);
                    }
                    if (gd >= 0.f)
                        for (int k = 0; k < d; ++k) P2[k * TCR + r] = -G[k * TCR + r];
                }
                float nrm = 0.f;
                bool fin = true;
                for (int k = 0; k < d; ++k) {
                    P1[k * TCR + r] = G[k * TCR + r];
                    const float dk = P2[k * TCR + r];
                    fin = fin && isfinite(dk);
                    nrm = fmaxf(nrm, fabsf(dk));
                }
                if (!fin) { bad = 1; stop = true; }
                else if (nrm == 0.f) { conv = stop = true; }
                else { dn = nrm; sig = (float)S.step / nrm; phase = 1; }
            } else {
                float s0 = 0.f, s1 = 0.f;
                for (int k = 0; k < d; ++k) {
                    s0 = fmaf(P1[k * TCR + r], P2[k * TCR + r], s0);
                    s1 = fmaf(G[k * TCR + r], P2[k * TCR + r], s1);
                }
                const float curv = (s1 - s0) / sig;
                float al = (curv > 0.f) ? -s0 / curv : sig;
                const float cap = (float)S.step_max / dn;
                if (al > cap) al = cap;
                ++it;
                if (!isfinite(al)) { bad = 1; stop = true; }
                else {
                    for (int k = 0; k < d; ++k) V[k * TCR + r] = fmaf(al, P2[k * TCR + r], V[k * TCR + r]);
                    if (al * dn < (float)S.eps) conv = stop = true;
                    phase = 0;
                }
            }
            if (it >= S.max_iters) stop = true;
            if (stop) active = false;
        }
        if (aborted) break;
        // certificate at the final v in fp32 (forward pass only)
        if (lead)
            for (int k = 0; k < d; ++k) PT[k * TCR + r] = V[k * TCR + r];
        if (!tile_eval(T, a, false, X, PT, G, ybuf, io, nmax, s_red)) break;
        if (valid && lead) {
            n_it += it;
            n_pairs++;
            n_sumN += N;
            n_cert += io.N;
            const int cap = (!conv && !bad) ? 1 : 0;
            for (int k = 0; k < d; ++k) a.D.vfin[pid * a.ld + k] = V[k * TCR + r];
            a.D.iters[pid] = it;
            a.D.flags[pid] = (uint8_t)(cap | (bad << 1));
            const float F = io.F, rr = io.resid;
            const bool fin = isfinite(F) && isfinite(rr) && io.N > 0;
            uint8_t pass;
            if (!fin) pass = 0;
            else if ((double)rr < CERT_BAND_LO * a.D.tol) pass = 1;
            else if ((double)rr > CERT_BAND_HI * a.D.tol) pass = 0;
            else pass = 2;
            a.D.pF[pid] = (double)F;
            a.D.pR[pid] = (double)rr;
            a.D.pP[pid] = pass;
            if (pass == 2) {
                const int pos = atomicAdd(a.D.amb_count + a.D.problem, 1);
                a.D.amb_wl[begin + pos] = (int32_t)pid;
            }
        }
    }
    if (T.abort && tid == 0) atomicExch(a.err, 1);
    if (MODE == LQ_DESC && a.D.stats && lead) {
        atomicAdd(a.D.stats + 0, n_it);
        atomicAdd(a.D.stats + 2, n_g);
        atomicAdd(a.D.stats + 3, n_rk);
        atomicAdd(a.D.stats + 4, n_adj);
        atomicAdd(a.D.stats + 5, n_pairs);
        atomicAdd(a.D.stats + 6, n_sumN);
        atomicAdd(a.D.stats + 7, n_cert);
    }
    // free the tensor memory (after every product has completed or timed out)
    fence_before();
    __syncthreads();
    fence_after();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(T.tm), "r"(TM_COLS));
}

// ---------------------------------------------------------------------------
// Host side.
// ---------------------------------------------------------------------------
namespace {

uint16_t bf16_rn(float f)
{
    uint32_t u;
    std::memcpy(&u, &f, 4);
    u += 0x7FFFu + ((u >> 16) & 1u);
    return (uint16_t)(u >> 16);
}
float bf16_val(uint16_t b)
{
    uint32_t u = (uint32_t)b << 16;
    float f;
    std::memcpy(&f, &u, 4);
    return f;
}
size_t host_off(int r, int k, int kc) { return (size_t)(r >> 3) * (kc >> 3) * 128 + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2; }

// Splits a rows x kc matrix (double, row-major) into bf16 hi/lo in the
// core-matrix layout.
void pack_split(const std::vector<double> &W, int rows, int kc, std::vector<uint8_t> &hi, std::vector<uint8_t> &lo)
{
    hi.assign((size_t)rows * kc * 2, 0);
    lo.assign((size_t)rows * kc * 2, 0);
    for (int r = 0; r < rows; ++r)
        for (int k = 0; k < kc; ++k) {
            const double w = W[(size_t)r * kc + k];
            const uint16_t h = bf16_rn((float)w);
            const uint16_t l = bf16_rn((float)(w - (double)bf16_val(h)));
            std::memcpy(&hi[host_off(r, k, kc)], &h, 2);
            std::memcpy(&lo[host_off(r, k, kc)], &l, 2);
        }
}

}  // namespace

bool lq_tc_geometry(int d, int m, LqTcGeom *g)
{
    g->d = d;
    g->m = m;
    g->dp = (d + 15) / 16 * 16;
    g->mp = (m + 15) / 16 * 16;
    const int dp = g->dp, mp = g->mp;
    g->KZ = 2 * dp + mp;
    g->KV = g->KZ;
    // one dense product per pass (wide N keeps each MMA at full rate):
    // forward (k_gamma, k_p, y) from (gamma, p); reverse (r_gamma, r_p) from (w_gamma, w_p, b y)
    g->fwd[0] = LqTcProd{0, 0, 2 * dp, 0, 2 * dp + mp, 2 * dp};
    g->fwd[1] = g->fwd[0];
    g->rev[0] = LqTcProd{0, 0, 2 * dp + mp, 0, 2 * dp, 2 * dp + mp};
    g->rev[1] = g->rev[0];
    g->w_bytes = (size_t)(2 * dp + mp) * 2 * dp * 2;
    g->z_bytes = (size_t)TCR * g->KZ * 2;
    g->smem = 2 * g->w_bytes + 2 * g->z_bytes;
    // N = 2 dp + mp <= 256 in one MMA, the accumulator and 4 dp state
    // columns within 512 TMEM columns, shared memory within budget
    return dp <= 64 && 2 * dp + mp <= 256 && g->smem <= LQ_TC_SMEM_MAX;
}

void lq_tc_matrices(const LqTcGeom &g, const double *A, const double *B, std::vector<uint8_t> &wf_hi,
                    std::vector<uint8_t> &wf_lo, std::vector<uint8_t> &wv_hi, std::vector<uint8_t> &wv_lo)
{
    const int d = g.d, m = g.m, dp = g.dp, mp = g.mp;
    const int kf = 2 * dp, nf = 2 * dp + mp, kv = 2 * dp + mp, nv = 2 * dp;
    std::vector<double> C((size_t)d * d, 0.0);
    for (int i = 0; i < d; ++i)
        for (int j = 0; j < d; ++j) {
            double s = 0;
            for (int k = 0; k < m; ++k) s += B[(size_t)i * m + k] * B[(size_t)j * m + k];
            C[(size_t)i * d + j] = s;
        }
    // forward: rows (k_gamma | k_p | y), columns (gamma | p)
    std::vector<double> Wf((size_t)nf * kf, 0.0);
    for (int j = 0; j < d; ++j)
        for (int k = 0; k < d; ++k) {
            Wf[(size_t)j * kf + k] = -A[(size_t)j * d + k];
            Wf[(size_t)j * kf + dp + k] = -C[(size_t)j * d + k];
            Wf[(size_t)(dp + j) * kf + dp + k] = A[(size_t)k * d + j];
        }
    for (int l = 0; l < m; ++l)
        for (int k = 0; k < d; ++k) Wf[(size_t)(2 * dp + l) * kf + dp + k] = B[(size_t)k * m + l];
    // reverse: rows (r_gamma | r_p), columns (w_gamma | w_p | b y)
    std::vector<double> Wv((size_t)nv * kv, 0.0);
    for (int j = 0; j < d; ++j)
        for (int k = 0; k < d; ++k) {
            Wv[(size_t)j * kv + k] = -A[(size_t)k * d + j];
            Wv[(size_t)(dp + j) * kv + k] = -C[(size_t)j * d + k];
            Wv[(size_t)(dp + j) * kv + dp + k] = A[(size_t)j * d + k];
        }
    for (int i = 0; i < d; ++i)
        for (int l = 0; l < m; ++l) Wv[(size_t)(dp + i) * kv + 2 * dp + l] = B[(size_t)i * m + l];
    pack_split(Wf, nf, kf, wf_hi, wf_lo);
    pack_split(Wv, nv, kv, wv_hi, wv_lo);
}

size_t lq_tc_vec_slot(const LqTcGeom &g) { return (size_t)6 * g.dp * TCR; }
size_t lq_tc_ybuf_slot(const LqTcGeom &g) { return (size_t)MAX_N * 4 * g.mp * TCR; }

// The dynamic shared-memory limit of each kernel is raised once per device
// (raising it again while an instance runs on another stream would wait for
// that instance).
static size_t g_smem_set[64][3];

template <int MODE>
static cudaError_t launch_mode(const LqTcArgs &a, int grid, size_t smem, cudaStream_t s)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (smem > g_smem_set[dev][MODE]) {
        e = cudaFuncSetAttribute(k_lq_tc<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)LQ_TC_SMEM_MAX);
        if (e != cudaSuccess) return e;
        g_smem_set[dev][MODE] = LQ_TC_SMEM_MAX;
    }
    k_lq_tc<MODE><<<grid, TCT, smem, s>>>(a);
    return cudaGetLastError();
}

cudaError_t lq_tc_launch(int mode, const LqTcArgs &a, int grid, size_t smem, cudaStream_t s)
{
    if (smem > LQ_TC_SMEM_MAX) return cudaErrorInvalidValue;
    switch (mode) {
    case LQ_ROWS_EVAL: return launch_mode<LQ_ROWS_EVAL>(a, grid, smem, s);
    case LQ_ROWS_GRAD: return launch_mode<LQ_ROWS_GRAD>(a, grid, smem, s);
    default: return launch_mode<LQ_DESC>(a, grid, smem, s);
    }
}

}  // namespace hjd
