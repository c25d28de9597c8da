// SVRG inner loop (Sec. 2.3, SVRGsolve): m serial variance-reduced steps
//   r = x_i^T (W - Wt),  W <- W - eta [lambda (W - Wt) - c_i x_i r + M]
// (or, with a batch of b samples, the stochastic term averaged over b)
// on the p columns of W, which are independent chains sharing the sampled
// index sequence.  One CTA owns PC columns and the whole d-long state of each:
// the difference Delta = W - Wt and the anchor gradient M live in registers,
// the sampled columns x_i stream through a 4-deep shared-memory ring filled by
// cp.async three steps ahead (the index sequence is known in advance), and
// x_i^T Delta is reduced with warp shuffles and one barrier per step.
#include <cuda_bf16.h>

#include <algorithm>
#include <type_traits>
#include <cstdlib>
#include <string>

#include "kernels.cuh"

namespace lra {

namespace {

constexpr int kRing = 4;

template <int BYTES>
__device__ __forceinline__ void cp_async_bytes(void *smem, const void *gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    if constexpr (BYTES == 16)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem));
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(sa), "l"(gmem), "n"(BYTES));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

// One sample per step on a single warp (d <= 512), two steps per iteration.
// With Delta_{t+1} = a Delta_t + c_t x_t - eta M (a = 1 - eta lambda,
// c_t = eta c_{i_t} r_t), the next step's r follows from dot products that do
// not wait for c_t:
//   r_{t+1} = a x_{t+1}^T Delta_t + c_t x_{t+1}^T x_t - x_{t+1}^T (eta M),
// so the reduction for step t + 1 and the one for step t + 2 (taken on
// Delta_{t+1} once c_t is known) run together, and the serial chain per step
// is about half the dot-and-shuffle latency.  Lane l owns rows 4 (l + 32 s) + v.
// The ring holds 8 columns, fetched 7 steps ahead.
template <typename TX, int S, int PC>
__global__ void __launch_bounds__(32) svrg_inner_pair_kernel(
    const TX *__restrict__ X, int64_t ldx, int64_t dpad, int p, float *__restrict__ W,
    const float *__restrict__ Wt, const float *__restrict__ M, const int32_t *__restrict__ idx,
    const float *__restrict__ cval, int64_t m, float eta, float lam,
    float etac) {
    constexpr int R = 8;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    TX *ring = reinterpret_cast<TX *>(smem_raw);  // [R][dpad]
    const int lane = threadIdx.x;
    const int j0 = blockIdx.x * PC;
    constexpr int BYTES = 4 * sizeof(TX);

    float dl[S][4][PC];   // Delta = W - Wt
    float mm[S][4][PC];   // eta * M
#pragma unroll
    for (int s = 0; s < S; ++s) {
        const int64_t r = 4 * ((int64_t)lane + 32 * s);
#pragma unroll
        for (int j = 0; j < PC; ++j) {
            const bool ok = (r < dpad) && (j0 + j < p);
            const int64_t off = r + (int64_t)(j0 + j) * dpad;
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                dl[s][v][j] = ok ? (W[off + v] - Wt[off + v]) : 0.0f;
                mm[s][v][j] = ok ? eta * M[off + v] : 0.0f;
            }
        }
    }

    auto prefetch = [&](int64_t t) {
        if (t < m) {
            const TX *col = X + (int64_t)idx[t] * ldx;
            TX *slot = ring + (t & (R - 1)) * dpad;
#pragma unroll
            for (int s = 0; s < S; ++s) {
                const int64_t r = 4 * ((int64_t)lane + 32 * s);
                if (r < dpad) cp_async_bytes<BYTES>(slot + r, col + r);
            }
        }
        cp_async_commit();
    };
    auto load = [&](int64_t t, float (&x)[S][4]) {
        const TX *slot = ring + (t & (R - 1)) * dpad;
#pragma unroll
        for (int s = 0; s < S; ++s) {
            const int64_t r = 4 * ((int64_t)lane + 32 * s);
            if (t < m && r < dpad) {
                load4_f32(slot + r, x[s]);
            } else {
#pragma unroll
                for (int v = 0; v < 4; ++v) x[s][v] = 0.0f;
            }
        }
    };
    // partial sums of y^T Delta, y^T (eta M) per column and y^T z
    auto dots = [&](const float (&y)[S][4], const float (&z)[S][4], float (&u)[PC], float (&w)[PC], float &vv) {
#pragma unroll
        for (int j = 0; j < PC; ++j) {
            float a0 = 0.0f, a1 = 0.0f;
#pragma unroll
            for (int s = 0; s < S; ++s)
#pragma unroll
                for (int v = 0; v < 4; ++v) {
                    a0 = fmaf(y[s][v], dl[s][v][j], a0);
                    a1 = fmaf(y[s][v], mm[s][v][j], a1);
                }
            u[j] = a0;
            w[j] = a1;
        }
        float a2 = 0.0f;
#pragma unroll
        for (int s = 0; s < S; ++s)
#pragma unroll
            for (int v = 0; v < 4; ++v) a2 = fmaf(y[s][v], z[s][v], a2);
        vv = a2;
    };
    auto update = [&](const float (&x)[S][4], const float (&c)[PC], float a) {
#pragma unroll
        for (int s = 0; s < S; ++s)
#pragma unroll
            for (int v = 0; v < 4; ++v)
#pragma unroll
                for (int j = 0; j < PC; ++j) dl[s][v][j] = fmaf(a, dl[s][v][j], fmaf(c[j], x[s][v], -mm[s][v][j]));
    };

#pragma unroll
    for (int u = 0; u < R - 1; ++u) prefetch(u);
    const float a = 1.0f - eta * lam;
    float x0[S][4], x1[S][4], x2[S][4];
    float r[PC];
    cp_async_wait<R - 2>();
    load(0, x0);
#pragma unroll
    for (int j = 0; j < PC; ++j) {
        float acc = 0.0f;
#pragma unroll
        for (int s = 0; s < S; ++s)
#pragma unroll
            for (int v = 0; v < 4; ++v) acc = fmaf(x0[s][v], dl[s][v][j], acc);
        r[j] = warp_sum(acc);
    }
    for (int64_t t = 0; t < m; t += 2) {
        prefetch(t + R - 1);
        prefetch(t + R);
        cp_async_wait<R - 2>();
        load(t + 1, x1);
        load(t + 2, x2);
        const float c0 = etac * cval[t];
        const float c1v = (t + 1 < m) ? etac * cval[t + 1] : 0.0f;
        float ct[PC];
#pragma unroll
        for (int j = 0; j < PC; ++j) ct[j] = c0 * r[j];
        // chain A: r_{t+1} from Delta_t
        float uA[PC], wA[PC], vA;
        dots(x1, x0, uA, wA, vA);
        // step t
        update(x0, ct, a);
        // chain B: r_{t+2} from Delta_{t+1}, less the c_{t+1} term
        float uB[PC], wB[PC], vB;
        dots(x2, x1, uB, wB, vB);
#pragma unroll
        for (int j = 0; j < PC; ++j) {
            uA[j] = warp_sum(uA[j]);
            wA[j] = warp_sum(wA[j]);
            uB[j] = warp_sum(uB[j]);
            wB[j] = warp_sum(wB[j]);
        }
        vA = warp_sum(vA);
        vB = warp_sum(vB);
        float c1[PC];
#pragma unroll
        for (int j = 0; j < PC; ++j) {
            const float r1 = fmaf(a, uA[j], fmaf(ct[j], vA, -wA[j]));
            c1[j] = c1v * r1;
        }
        if (t + 1 < m) {
            // step t + 1
            update(x1, c1, a);
#pragma unroll
            for (int j = 0; j < PC; ++j) r[j] = fmaf(a, uB[j], fmaf(c1[j], vB, -wB[j]));
        }
#pragma unroll
        for (int s = 0; s < S; ++s)
#pragma unroll
            for (int v = 0; v < 4; ++v) x0[s][v] = x2[s][v];
    }
    cp_async_wait<0>();
#pragma unroll
    for (int s = 0; s < S; ++s) {
        const int64_t r0 = 4 * ((int64_t)lane + 32 * s);
#pragma unroll
        for (int j = 0; j < PC; ++j) {
            if (r0 < dpad && j0 + j < p) {
                const int64_t off = r0 + (int64_t)(j0 + j) * dpad;
#pragma unroll
                for (int v = 0; v < 4; ++v) W[off + v] = Wt[off + v] + dl[s][v][j];
            }
        }
    }
}

// One sample per step.  Thread t owns rows 4 (t + s NT) + v for s < S, v < 4
// (rows >= dpad skipped).
template <typename TX, int S, int PC>
__global__ void __launch_bounds__(512) svrg_inner1_kernel(
    const TX *__restrict__ X, int64_t ldx, int64_t dpad, int p, float *__restrict__ W,
    const float *__restrict__ Wt, const float *__restrict__ M, const int32_t *__restrict__ idx,
    const float *__restrict__ cval, int64_t m, float eta, float lam,
    float etac) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    TX *ring = reinterpret_cast<TX *>(smem_raw);  // [kRing][dpad]
    __shared__ float red[2][16][PC];

    const int tid = threadIdx.x;
    const int NT = blockDim.x;
    const int lane = tid & 31, warp = tid >> 5, nwarps = NT >> 5;
    const int j0 = blockIdx.x * PC;
    constexpr int BYTES = 4 * sizeof(TX);

    float dl[S][4][PC];   // Delta = W - Wt
    float mm[S][4][PC];   // eta * M
#pragma unroll
    for (int s = 0; s < S; ++s) {
        const int64_t r = 4 * ((int64_t)tid + (int64_t)s * NT);
#pragma unroll
        for (int j = 0; j < PC; ++j) {
            const bool ok = (r < dpad) && (j0 + j < p);
            const int64_t off = r + (int64_t)(j0 + j) * dpad;
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                dl[s][v][j] = ok ? (W[off + v] - Wt[off + v]) : 0.0f;
                mm[s][v][j] = ok ? eta * M[off + v] : 0.0f;
            }
        }
    }

    auto prefetch = [&](int64_t t) {
        if (t < m) {
            const int64_t i = idx[t];
            const TX *col = X + i * ldx;
            TX *slot = ring + (t & (kRing - 1)) * dpad;
#pragma unroll
            for (int s = 0; s < S; ++s) {
                const int64_t r = 4 * ((int64_t)tid + (int64_t)s * NT);
                if (r < dpad) cp_async_bytes<BYTES>(slot + r, col + r);
            }
        }
        cp_async_commit();
    };

    prefetch(0);
    prefetch(1);
    prefetch(2);
    const float a = 1.0f - eta * lam;

    for (int64_t t = 0; t < m; ++t) {
        prefetch(t + 3);
        cp_async_wait<3>();
        const TX *slot = ring + (t & (kRing - 1)) * dpad;
        float x[S][4];
#pragma unroll
        for (int s = 0; s < S; ++s) {
            const int64_t r = 4 * ((int64_t)tid + (int64_t)s * NT);
            if (r < dpad) {
                load4_f32(slot + r, x[s]);
            } else {
#pragma unroll
                for (int v = 0; v < 4; ++v) x[s][v] = 0.0f;
            }
        }
        const float ci = cval[t];
        float part[PC];
#pragma unroll
        for (int j = 0; j < PC; ++j) {
            float acc = 0.0f;
#pragma unroll
            for (int s = 0; s < S; ++s)
#pragma unroll
                for (int v = 0; v < 4; ++v) acc = fmaf(x[s][v], dl[s][v][j], acc);
            part[j] = warp_sum(acc);
        }
        float coef[PC];
        if (nwarps == 1) {
            // one warp: every lane already holds the full sum (no barrier)
#pragma unroll
            for (int j = 0; j < PC; ++j) coef[j] = etac * ci * part[j];
        } else {
            const int buf = (int)(t & 1);
            if (lane == 0) {
#pragma unroll
                for (int j = 0; j < PC; ++j) red[buf][warp][j] = part[j];
            }
            __syncthreads();
#pragma unroll
            for (int j = 0; j < PC; ++j) {
                float rj = 0.0f;
                for (int w = 0; w < nwarps; ++w) rj += red[buf][w][j];
                coef[j] = etac * ci * rj;
            }
        }
#pragma unroll
        for (int s = 0; s < S; ++s)
#pragma unroll
            for (int v = 0; v < 4; ++v)
#pragma unroll
                for (int j = 0; j < PC; ++j)
                    dl[s][v][j] = fmaf(a, dl[s][v][j], fmaf(coef[j], x[s][v], -mm[s][v][j]));
    }
    cp_async_wait<0>();

#pragma unroll
    for (int s = 0; s < S; ++s) {
        const int64_t r = 4 * ((int64_t)tid + (int64_t)s * NT);
#pragma unroll
        for (int j = 0; j < PC; ++j) {
            if (r < dpad && j0 + j < p) {
                const int64_t off = r + (int64_t)(j0 + j) * dpad;
#pragma unroll
                for (int v = 0; v < 4; ++v) W[off + v] = Wt[off + v] + dl[s][v][j];
            }
        }
    }
}

// One sample per step on NT = 32 NW threads (d > 512), two steps per block
// barrier.  With Delta_{t+1} = a Delta_t + c_t x_t - eta M, the look-ahead
// identity of svrg_inner_pair_kernel,
//   r_{t+1} = a x_{t+1}^T Delta_t + c_t x_{t+1}^T x_t - x_{t+1}^T (eta M),
// lets the dot products of steps t + 1 and t + 2 (the latter taken on
// Delta_{t+1} once c_t is known, less its c_{t+1} term) share one block
// reduction.  The kernel is bound by instruction issue, so it is written to
// issue few: the per-thread dot products and the updates of Delta run on
// packed FP32x2 FMAs (fma.rn.f32x2: two independent round-to-nearest FMAs,
// the same values as two fmaf), a warp reduces its NV partial sums with a
// transposing butterfly (NP/2 + NP/4 + ... exchanges instead of 5 per value),
// and the NV totals are then summed over the warps from a shared row of 16
// (zero for absent warps).  Thread t owns rows 4 (t + s NT) + v; the ring
// holds R columns, fetched R - 1 steps ahead, and each thread copies and reads
// only its own rows of them.
__device__ __forceinline__ float2 ffma2(float2 a, float2 b, float2 c) {
    uint64_t d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;"
        : "=l"(d)
        : "l"(*reinterpret_cast<const uint64_t *>(&a)), "l"(*reinterpret_cast<const uint64_t *>(&b)),
          "l"(*reinterpret_cast<const uint64_t *>(&c)));
    return *reinterpret_cast<float2 *>(&d);
}

// Warp sums of NP values (NP a power of two, 2 <= NP <= 32): after the call
// lane l holds the warp total of value l >> (5 - log2 NP).  Level o = 16, 8, ...
// halves the values a lane keeps (the upper lanes keep the upper half) while
// adding the partner's copy; the last levels add within each group of 32 / NP
// lanes.  Fixed order, so the result does not depend on timing.
template <int NP>
__device__ __forceinline__ float warp_transpose_sum(float (&v)[NP], int lane) {
    int cnt = NP;
#pragma unroll
    for (int o = 16; o >= 32 / NP; o >>= 1) {
        const int half = cnt >> 1;
        const bool upper = (lane & o) != 0;
#pragma unroll
        for (int i = 0; i < NP / 2; ++i) {
            if (i < half) {
                const float send = upper ? v[i] : v[i + half];
                const float keep = upper ? v[i + half] : v[i];
                v[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
            }
        }
        cnt = half;
    }
    float r = v[0];
#pragma unroll
    for (int o = 16 / NP; o > 0; o >>= 1) r += __shfl_xor_sync(0xffffffffu, r, o);
    return r;
}

// Block totals of NV values over NW <= 16 warps: warp totals by the
// transposing butterfly, one shared row of 16 per value; then NW lanes per
// value read its warps' entries and sum them by an xor butterfly, and every
// lane takes the totals by shuffles.  The tree is fixed (pairs, then pairs of
// pairs), so the result does not depend on timing; entries of absent warps
// hold zeros.
template <int NV, int NP, int NW>
__device__ __forceinline__ void block_sum16(float (&v)[NP], float (*red)[16], int lane, int warp) {
    constexpr int LB = 5 - (NP == 2 ? 1 : NP == 4 ? 2 : NP == 8 ? 3 : NP == 16 ? 4 : 5);
    const float w = warp_transpose_sum<NP>(v, lane);
    const int idx = lane >> LB;
    if ((lane & ((1 << LB) - 1)) == 0 && idx < NV) red[idx][warp] = w;
    __syncthreads();
    constexpr int G = NW <= 2 ? 2 : NW <= 4 ? 4 : NW <= 8 ? 8 : 16;  // lanes per value
    constexpr int VPR = 32 / G;                                       // values per round
    constexpr int RND = (NV + VPR - 1) / VPR;
    float part[RND];
#pragma unroll
    for (int rr = 0; rr < RND; ++rr) {
        const int i = rr * VPR + lane / G;
        part[rr] = i < NV ? red[i][lane % G] : 0.0f;
    }
#pragma unroll
    for (int o = 1; o < G; o <<= 1)
#pragma unroll
        for (int rr = 0; rr < RND; ++rr) part[rr] += __shfl_xor_sync(0xffffffffu, part[rr], o);
#pragma unroll
    for (int i = 0; i < NV; ++i) v[i] = __shfl_sync(0xffffffffu, part[i / VPR], (i % VPR) * G);
}

// Ring depth of the look-ahead kernel: the deepest of 8, 6, 4, 3 columns of
// up to 2048 S rows that fits the shared-memory budget.
template <typename TX, int S>
__host__ __device__ constexpr int la_ring() {
    constexpr size_t col = (size_t)2048 * S * sizeof(TX);
    return 8 * col <= 220 * 1024 ? 8 : 6 * col <= 220 * 1024 ? 6 : 4 * col <= 220 * 1024 ? 4 : 3;
}

template <int NV>
__host__ __device__ constexpr int pow2_at_least() { return NV <= 2 ? 2 : NV <= 4 ? 4 : NV <= 8 ? 8 : NV <= 16 ? 16 : 32; }

template <typename TX, int S, int PC, int NW, int R = la_ring<TX, S>()>
__global__ void __launch_bounds__(32 * NW) svrg_inner_la_kernel(
    const TX *__restrict__ X, int64_t ldx, int64_t dpad, int p, float *__restrict__ W,
    const float *__restrict__ Wt, const float *__restrict__ M, const int32_t *__restrict__ idx,
    const float *__restrict__ cval, int64_t m, float eta, float lam,
    float etac) {
    constexpr int NV = 4 * PC + 2;  // uA, wA, uB, wB per column, then vA, vB
    constexpr int NP = pow2_at_least<NV>();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    TX *ring = reinterpret_cast<TX *>(smem_raw);  // [R][dpad]
    __shared__ __align__(16) float red[3][NV][16];

    const int tid = threadIdx.x;
    const int NT = blockDim.x;
    const int lane = tid & 31, warp = tid >> 5;
    const int j0 = blockIdx.x * PC;
    constexpr int BYTES = 4 * sizeof(TX);

    for (int e = tid; e < 3 * NV * 16; e += NT) (&red[0][0][0])[e] = 0.0f;
    // the sample indices and weights in windows of 128 steps, two in shared memory:
    // window w in slot w & 1, window w + 1 fetched while w runs (NT >= 128 here)
    __shared__ int32_t sidx[2][128];
    __shared__ float scv[2][128];
    if (tid < 128) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int64_t u = (int64_t)h * 128 + tid;
            sidx[h][tid] = u < m ? idx[u] : 0;
            scv[h][tid] = u < m ? cval[u] : 0.0f;
        }
    }
    // every zero and window entry lands before any warp reads it
    __syncthreads();

    // Delta = W - Wt and -eta M, rows 4 (t + s NT) + {0, 1} and + {2, 3} as pairs
    // (-eta M is kept negated, so every update is two packed FMAs)
    float2 dl[S][2][PC];
    float2 mm[S][2][PC];
#pragma unroll
    for (int s = 0; s < S; ++s) {
        const int64_t r = 4 * ((int64_t)tid + (int64_t)s * NT);
#pragma unroll
        for (int j = 0; j < PC; ++j) {
            const bool ok = (r < dpad) && (j0 + j < p);
            const int64_t off = r + (int64_t)(j0 + j) * dpad;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                dl[s][h][j] = ok ? make_float2(W[off + 2 * h] - Wt[off + 2 * h], W[off + 2 * h + 1] - Wt[off + 2 * h + 1])
                                 : make_float2(0.0f, 0.0f);
                mm[s][h][j] = ok ? make_float2(-eta * M[off + 2 * h], -eta * M[off + 2 * h + 1]) : make_float2(0.0f, 0.0f);
            }
        }
    }

    // rows of this thread and ring slots in 32-bit arithmetic (dpad <= 8192 here);
    // column t sits in slot t mod R
    const int dp = (int)dpad;
    int rofs[S];
#pragma unroll
    for (int s = 0; s < S; ++s) rofs[s] = 4 * (tid + s * NT);
    auto prefetch = [&](int64_t t, int slot) {
        if (t < m) {
            const TX *col = X + (int64_t)sidx[(t >> 7) & 1][t & 127] * ldx;
            TX *dst = ring + slot * dp;
#pragma unroll
            for (int s = 0; s < S; ++s)
                if (rofs[s] < dp) cp_async_bytes<BYTES>(dst + rofs[s], col + rofs[s]);
        }
        cp_async_commit();
    };
    auto load = [&](int64_t t, int slot_i, float2 (&x)[S][2]) {
        const TX *slot = ring + slot_i * dp;
#pragma unroll
        for (int s = 0; s < S; ++s) {
            const int r = rofs[s];
            if (t < m && r < dp) {
                float q[4];
                load4_f32(slot + r, q);
                x[s][0] = make_float2(q[0], q[1]);
                x[s][1] = make_float2(q[2], q[3]);
            } else {
                x[s][0] = make_float2(0.0f, 0.0f);
                x[s][1] = make_float2(0.0f, 0.0f);
            }
        }
    };
    // partial sums of y^T Delta and y^T (-eta M) per column, and y^T z
    auto dots = [&](const float2 (&y)[S][2], const float2 (&z)[S][2], float *u, float *w, float &vv) {
#pragma unroll
        for (int j = 0; j < PC; ++j) {
            float2 a0 = make_float2(0.0f, 0.0f), a1 = make_float2(0.0f, 0.0f);
#pragma unroll
            for (int s = 0; s < S; ++s)
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    a0 = ffma2(y[s][h], dl[s][h][j], a0);
                    a1 = ffma2(y[s][h], mm[s][h][j], a1);
                }
            u[j] = a0.x + a0.y;
            w[j] = a1.x + a1.y;
        }
        float2 a2 = make_float2(0.0f, 0.0f);
#pragma unroll
        for (int s = 0; s < S; ++s)
#pragma unroll
            for (int h = 0; h < 2; ++h) a2 = ffma2(y[s][h], z[s][h], a2);
        vv = a2.x + a2.y;
    };
    const float a = 1.0f - eta * lam;
    const float2 a2v = make_float2(a, a);
    auto update = [&](const float2 (&x)[S][2], const float (&c)[PC]) {
#pragma unroll
        for (int s = 0; s < S; ++s)
#pragma unroll
            for (int h = 0; h < 2; ++h)
#pragma unroll
                for (int j = 0; j < PC; ++j)
                    dl[s][h][j] = ffma2(a2v, dl[s][h][j], ffma2(make_float2(c[j], c[j]), x[s][h], mm[s][h][j]));
    };

#pragma unroll
    for (int u = 0; u < R - 1; ++u) prefetch(u, u);
    float2 x0[S][2], x1[S][2], x2[S][2];
    float r[PC];
    cp_async_wait<R - 2>();
    load(0, 0, x0);
    {
        constexpr int NP0 = pow2_at_least<PC>();
        float v0[NP0];
#pragma unroll
        for (int i = 0; i < NP0; ++i) v0[i] = 0.0f;
#pragma unroll
        for (int j = 0; j < PC; ++j) {
            float2 acc = make_float2(0.0f, 0.0f);
#pragma unroll
            for (int s = 0; s < S; ++s)
#pragma unroll
                for (int h = 0; h < 2; ++h) acc = ffma2(x0[s][h], dl[s][h][j], acc);
            v0[j] = acc.x + acc.y;
        }
        block_sum16<PC, NP0, NW>(v0, red[2], lane, warp);
#pragma unroll
        for (int j = 0; j < PC; ++j) r[j] = v0[j];
    }
    int s0 = 0;  // t mod R
    int32_t pidx = 0;  // the next window's entry of this thread, between load and store
    float pcv = 0.0f;
    // two steps from column t in xa (columns t + 1, t + 2 loaded into xb, xc);
    // the loop alternates the roles of x0 and x2 instead of copying x2 to x0
    auto two_steps = [&](int64_t t, float2 (&xa)[S][2], float2 (&xb)[S][2], float2 (&xc)[S][2],
                         float (*redb)[16]) {
        const int sm1 = s0 == 0 ? R - 1 : s0 - 1;
        const int sp1 = s0 + 1 >= R ? s0 + 1 - R : s0 + 1;
        const int sp2 = s0 + 2 >= R ? s0 + 2 - R : s0 + 2;
        prefetch(t + R - 1, sm1);
        prefetch(t + R, s0);
        cp_async_wait<R - 2>();
        load(t + 1, sp1, xb);
        load(t + 2, sp2, xc);
        s0 = sp2;
        // window (t / 128) + 1: loaded into registers at t = 0 mod 128 and stored
        // two steps later; its slot last served window t / 128 - 1, whose final
        // reads came before the previous block barrier, and its first reads come
        // ~60 barriers later
        if ((t & 127) == 0) {
            const int64_t u = t + 128 + tid;
            if (tid < 128) {
                pidx = u < m ? idx[u] : 0;
                pcv = u < m ? cval[u] : 0.0f;
            }
        } else if ((t & 127) == 2 && tid < 128) {
            sidx[((t >> 7) + 1) & 1][tid] = pidx;
            scv[((t >> 7) + 1) & 1][tid] = pcv;
        }
        const float c0 = etac * scv[(t >> 7) & 1][t & 127];
        const float c1v = (t + 1 < m) ? etac * scv[((t + 1) >> 7) & 1][(t + 1) & 127] : 0.0f;
        float ct[PC];
#pragma unroll
        for (int j = 0; j < PC; ++j) ct[j] = c0 * r[j];
        float acc[NP];
#pragma unroll
        for (int i = NV; i < NP; ++i) acc[i] = 0.0f;
        // chain A: r_{t+1} from Delta_t
        dots(xb, xa, acc, acc + PC, acc[4 * PC]);
        // step t
        update(xa, ct);
        // chain B: r_{t+2} from Delta_{t+1}, less the c_{t+1} term
        dots(xc, xb, acc + 2 * PC, acc + 3 * PC, acc[4 * PC + 1]);
        block_sum16<NV, NP, NW>(acc, redb, lane, warp);
        float c1[PC];
#pragma unroll
        for (int j = 0; j < PC; ++j) c1[j] = c1v * fmaf(a, acc[j], fmaf(ct[j], acc[4 * PC], acc[PC + j]));
        if (t + 1 < m) {
            // step t + 1
            update(xb, c1);
#pragma unroll
            for (int j = 0; j < PC; ++j)
                r[j] = fmaf(a, acc[2 * PC + j], fmaf(c1[j], acc[4 * PC + 1], acc[3 * PC + j]));
        }
    };
    for (int64_t t = 0; t < m; t += 4) {
        two_steps(t, x0, x1, x2, red[0]);
        if (t + 2 < m) two_steps(t + 2, x2, x1, x0, red[1]);
    }
    cp_async_wait<0>();

#pragma unroll
    for (int s = 0; s < S; ++s) {
        const int64_t r0 = 4 * ((int64_t)tid + (int64_t)s * NT);
#pragma unroll
        for (int j = 0; j < PC; ++j) {
            if (r0 < dpad && j0 + j < p) {
                const int64_t off = r0 + (int64_t)(j0 + j) * dpad;
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    W[off + 2 * h] = Wt[off + 2 * h] + dl[s][h][j].x;
                    W[off + 2 * h + 1] = Wt[off + 2 * h + 1] + dl[s][h][j].y;
                }
            }
        }
    }
}

// A batch of NB > 1 samples per step: the stochastic term averaged over the
// NB samples, every r_u taken at the same W.  One column per CTA; the ring
// holds D steps of NB columns, D - 1 steps fetched ahead; each thread copies
// and reads only its own rows of a column, so the ring needs no barrier.
template <typename TX, int S, int NB, int D>
__global__ void __launch_bounds__(512) svrg_inner_batch_kernel(
    const TX *__restrict__ X, int64_t ldx, int64_t dpad, int p, float *__restrict__ W,
    const float *__restrict__ Wt, const float *__restrict__ M, const int32_t *__restrict__ idx,
    const float *__restrict__ cval, int64_t m, float eta, float lam,
    float etac) {
    constexpr int PC = 1, MB = NB, nb = NB;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    TX *ring = reinterpret_cast<TX *>(smem_raw);  // [D * NB][dpad]
    __shared__ float red[2][16][NB];

    const int tid = threadIdx.x;
    const int NT = blockDim.x;
    const int lane = tid & 31, warp = tid >> 5, nwarps = NT >> 5;
    const int j0 = blockIdx.x * PC;
    constexpr int nslot = D * NB;  // a power of two
    constexpr int BYTES = 4 * sizeof(TX);

    float dl[S][4][PC];   // Delta = W - Wt
    float mm[S][4][PC];   // eta * M
#pragma unroll
    for (int s = 0; s < S; ++s) {
        const int64_t r = 4 * ((int64_t)tid + (int64_t)s * NT);
#pragma unroll
        for (int j = 0; j < PC; ++j) {
            const bool ok = (r < dpad) && (j0 + j < p);
            const int64_t off = r + (int64_t)(j0 + j) * dpad;
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                dl[s][v][j] = ok ? (W[off + v] - Wt[off + v]) : 0.0f;
                mm[s][v][j] = ok ? eta * M[off + v] : 0.0f;
            }
        }
    }

    auto prefetch = [&](int64_t t) {
        if (t < m) {
#pragma unroll
            for (int u = 0; u < NB; ++u) {
                const int64_t smp = t * NB + u;
                const TX *col = X + (int64_t)idx[smp] * ldx;
                TX *slot = ring + (smp & (nslot - 1)) * dpad;
#pragma unroll
                for (int s = 0; s < S; ++s) {
                    const int64_t r = 4 * ((int64_t)tid + (int64_t)s * NT);
                    if (r < dpad) cp_async_bytes<BYTES>(slot + r, col + r);
                }
            }
        }
        cp_async_commit();
    };
    auto load_x = [&](int64_t smp, float (&x)[S][4]) {
        const TX *slot = ring + (smp & (nslot - 1)) * dpad;
#pragma unroll
        for (int s = 0; s < S; ++s) {
            const int64_t r = 4 * ((int64_t)tid + (int64_t)s * NT);
            if (r < dpad) {
                load4_f32(slot + r, x[s]);
            } else {
#pragma unroll
                for (int v = 0; v < 4; ++v) x[s][v] = 0.0f;
            }
        }
    };

#pragma unroll
    for (int q = 0; q < D - 1; ++q) prefetch(q);
    const float a = 1.0f - eta * lam;
    const float invb = 1.0f / (float)nb;

    for (int64_t t = 0; t < m; ++t) {
        prefetch(t + D - 1);
        cp_async_wait<D - 1>();
        {
        // r_u = x_u^T Delta for every sample of the step (same Delta)
        float part[MB][PC];
#pragma unroll
        for (int u = 0; u < MB; ++u) {
            if (u < nb) {
                float x[S][4];
                load_x(t * nb + u, x);
#pragma unroll
                for (int j = 0; j < PC; ++j) {
                    float acc = 0.0f;
#pragma unroll
                    for (int s = 0; s < S; ++s)
#pragma unroll
                        for (int v = 0; v < 4; ++v) acc = fmaf(x[s][v], dl[s][v][j], acc);
                    part[u][j] = warp_sum(acc);
                }
            }
        }
        const int buf = (int)(t & 1);
        if (lane == 0) {
#pragma unroll
            for (int u = 0; u < MB; ++u)
                if (u < nb)
#pragma unroll
                    for (int j = 0; j < PC; ++j) red[buf][warp][u * PC + j] = part[u][j];
        }
        __syncthreads();
        float coef[MB][PC];
#pragma unroll
        for (int u = 0; u < MB; ++u) {
            if (u < nb) {
                const float cu = cval[t * nb + u];
#pragma unroll
                for (int j = 0; j < PC; ++j) {
                    float rj = 0.0f;
                    for (int w = 0; w < nwarps; ++w) rj += red[buf][w][u * PC + j];
                    coef[u][j] = etac * cu * rj * invb;
                }
            }
        }
        // Delta <- a Delta + sum_u coef_u x_u - eta M
        float upd[S][4][PC];
#pragma unroll
        for (int s = 0; s < S; ++s)
#pragma unroll
            for (int v = 0; v < 4; ++v)
#pragma unroll
                for (int j = 0; j < PC; ++j) upd[s][v][j] = -mm[s][v][j];
#pragma unroll
        for (int u = 0; u < MB; ++u) {
            if (u < nb) {
                float x[S][4];
                load_x(t * nb + u, x);
#pragma unroll
                for (int s = 0; s < S; ++s)
#pragma unroll
                    for (int v = 0; v < 4; ++v)
#pragma unroll
                        for (int j = 0; j < PC; ++j) upd[s][v][j] = fmaf(coef[u][j], x[s][v], upd[s][v][j]);
            }
        }
#pragma unroll
        for (int s = 0; s < S; ++s)
#pragma unroll
            for (int v = 0; v < 4; ++v)
#pragma unroll
                for (int j = 0; j < PC; ++j) dl[s][v][j] = fmaf(a, dl[s][v][j], upd[s][v][j]);
        }
    }
    cp_async_wait<0>();

#pragma unroll
    for (int s = 0; s < S; ++s) {
        const int64_t r = 4 * ((int64_t)tid + (int64_t)s * NT);
#pragma unroll
        for (int j = 0; j < PC; ++j) {
            if (r < dpad && j0 + j < p) {
                const int64_t off = r + (int64_t)(j0 + j) * dpad;
#pragma unroll
                for (int v = 0; v < 4; ++v) W[off + v] = Wt[off + v] + dl[s][v][j];
            }
        }
    }
}

template <typename TX, int S, int PC>
void launch_inner1(cudaStream_t st, const void *X, int64_t ldx, int64_t dpad, int p, float *W,
                   const float *Wt, const float *M, const int32_t *idx, const float *cval, int64_t m,
                   float eta, float lam, float etac, int nt) {
    auto k = svrg_inner1_kernel<TX, S, PC>;
    const size_t smem = (size_t)kRing * dpad * sizeof(TX);
    ensure_smem(k, (int)smem);
    const unsigned grid = (unsigned)ceil_div(p, PC);
    k<<<grid, nt, smem, st>>>((const TX *)X, ldx, dpad, p, W, Wt, M, idx, cval, m, eta, lam, etac);
    LRA_LAUNCHED();
}

template <typename TX, int S, int PC>
void launch_la(cudaStream_t st, const void *X, int64_t ldx, int64_t dpad, int p, float *W, const float *Wt,
               const float *M, const int32_t *idx, const float *cval, int64_t m, float eta, float lam, float etac, int nt) {
    constexpr int R = la_ring<TX, S>();
    const size_t smem = (size_t)R * dpad * sizeof(TX);
    auto go = [&](auto k) {
        ensure_smem(k, (int)smem);
        k<<<(unsigned)ceil_div(p, PC), nt, smem, st>>>((const TX *)X, ldx, dpad, p, W, Wt, M, idx, cval, m, eta, lam, etac);
        LRA_LAUNCHED();
    };
    if (nt <= 256)
        go(svrg_inner_la_kernel<TX, S, PC, 8, R>);
    else
        go(svrg_inner_la_kernel<TX, S, PC, 16, R>);
}

template <typename TX, int S, int NB, int D>
void launch_batch(cudaStream_t st, const void *X, int64_t ldx, int64_t dpad, int p, float *W,
                  const float *Wt, const float *M, const int32_t *idx, const float *cval, int64_t m,
                  float eta, float lam, float etac, int nt) {
    auto k = svrg_inner_batch_kernel<TX, S, NB, D>;
    const size_t smem = (size_t)D * NB * dpad * sizeof(TX);
    ensure_smem(k, (int)smem);
    k<<<(unsigned)p, nt, smem, st>>>((const TX *)X, ldx, dpad, p, W, Wt, M, idx, cval, m, eta, lam, etac);
    LRA_LAUNCHED();
}

template <typename TX>
constexpr size_t dt_size() { return sizeof(TX); }

constexpr size_t kRingBytes = 220 * 1024;

template <typename TX, int S, int PC>
void launch_pair(cudaStream_t st, const void *X, int64_t ldx, int64_t dpad, int p, float *W, const float *Wt,
                 const float *M, const int32_t *idx, const float *cval, int64_t m, float eta, float lam,
                 float etac) {
    auto k = svrg_inner_pair_kernel<TX, S, PC>;
    const size_t smem = (size_t)8 * dpad * sizeof(TX);
    ensure_smem(k, (int)smem);
    k<<<(unsigned)ceil_div(p, PC), 32, smem, st>>>((const TX *)X, ldx, dpad, p, W, Wt, M, idx, cval, m, eta, lam, etac);
    LRA_LAUNCHED();
}

template <typename TX>
void inner_dispatch(cudaStream_t st, const void *X, int64_t ldx, int64_t dpad, int p, float *W,
                    const float *Wt, const float *M, const int32_t *idx, const float *cval, int64_t m,
                    int nb, float eta, float lam, float etac) {
    // threads: 4 rows each, at most 512; S = row groups per thread.  Up to
    // d = 512 the one-sample step runs on a single warp (S <= 4): its x_i^T Delta
    // is then reduced by shuffles alone, without a block barrier per step
    const int64_t groups = dpad / 4;
    int nt = (int)std::min<int64_t>(512, round_up(groups, 32));
    int64_t S = ceil_div(groups, nt);
    if (nb == 1 && groups <= 128) {
        nt = 32;
        S = ceil_div(groups, 32);
    }
    if (S > 8) {
        set_error("dense inner loop supports d <= 16384");
        throw Error{LRA_EUNSUPPORTED};
    }
    if (nb == 1) {
        // columns per CTA: keep about <= 64 CTAs streaming the same x_i, and the
        // register state (8 S PC floats) within 64 registers
        const int pc = (p <= 64 || S > 4) ? 1 : 2;
        if ((size_t)kRing * dpad * (dt_size<TX>()) > kRingBytes) {
            set_error("dense inner loop: d too large for the shared-memory ring");
            throw Error{LRA_EUNSUPPORTED};
        }
        if (nt == 32) {
            // a single warp: two steps per iteration with the look-ahead identity
#define LRA_PAIR_CASE(SS, PCC)                                                                          \
    if (S == SS && pc == PCC) {                                                                         \
        launch_pair<TX, SS, PCC>(st, X, ldx, dpad, p, W, Wt, M, idx, cval, m, eta, lam, etac);               \
        return;                                                                                         \
    }
            LRA_PAIR_CASE(1, 1)
            LRA_PAIR_CASE(1, 2)
            LRA_PAIR_CASE(2, 1)
            LRA_PAIR_CASE(2, 2)
            LRA_PAIR_CASE(3, 1)
            LRA_PAIR_CASE(3, 2)
            LRA_PAIR_CASE(4, 1)
            LRA_PAIR_CASE(4, 2)
#undef LRA_PAIR_CASE
        }
        // several warps: two steps per block barrier (look-ahead identity); the
        // three column buffers of that kernel leave room for two columns per
        // CTA only up to two row groups per thread
        // the kernel is bound by instruction issue: 8 warps (four row groups
        // per thread) up to d = 4096 issue fewer reduction instructions per step
        // than 16 (measured 594 against 716 ns per step at d = 4096, p = 40);
        // beyond, the register state of four groups caps the threads at 512
        if (groups > 256 && groups <= 1024) {
            nt = 256;
            S = ceil_div(groups, nt);
        }
        const int pcl = (p <= 64 || S > 2) ? 1 : 2;
#define LRA_LA_CASE(SS, PCC)                                                                    \
    if (S == SS && pcl == PCC) {                                                                \
        launch_la<TX, SS, PCC>(st, X, ldx, dpad, p, W, Wt, M, idx, cval, m, eta, lam, etac, nt);     \
        return;                                                                                 \
    }
        LRA_LA_CASE(1, 1)
        LRA_LA_CASE(1, 2)
        LRA_LA_CASE(2, 1)
        LRA_LA_CASE(2, 2)
        LRA_LA_CASE(3, 1)
        LRA_LA_CASE(4, 1)
#undef LRA_LA_CASE
        // d > 8192: the look-ahead kernel's three column buffers would spill;
        // one barrier per step
        if (S <= 6) {
            launch_inner1<TX, 6, 1>(st, X, ldx, dpad, p, W, Wt, M, idx, cval, m, eta, lam, etac, nt);
        } else {
            launch_inner1<TX, 8, 1>(st, X, ldx, dpad, p, W, Wt, M, idx, cval, m, eta, lam, etac, nt);
        }
        return;
    }
    // a batch: one column per CTA; the ring holds four steps of nb columns when
    // it fits (three steps fetched ahead), else two
    const size_t col = (size_t)dpad * dt_size<TX>();
    const int depth = (size_t)4 * nb * col <= kRingBytes ? 4 : ((size_t)2 * nb * col <= kRingBytes ? 2 : 0);
    if (depth == 0) {
        set_error("dense inner loop: batch too large for d (the ring holds 2 b columns of X)");
        throw Error{LRA_EUNSUPPORTED};
    }
    if (S > 2 && nb > 8) {
        set_error("dense inner loop: batch 16 needs d <= 2048");
        throw Error{LRA_EUNSUPPORTED};
    }
    if (S == 3) S = 4;
    if (S > 4) S = 8;
    if (S == 8 && nb > 2) {
        set_error("dense inner loop: batch above 2 needs d <= 8192");
        throw Error{LRA_EUNSUPPORTED};
    }
    auto go = [&](auto sc, auto nbc) {
        constexpr int SS = decltype(sc)::value, NBB = decltype(nbc)::value;
        if (depth == 4)
            launch_batch<TX, SS, NBB, 4>(st, X, ldx, dpad, p, W, Wt, M, idx, cval, m, eta, lam, etac, nt);
        else
            launch_batch<TX, SS, NBB, 2>(st, X, ldx, dpad, p, W, Wt, M, idx, cval, m, eta, lam, etac, nt);
    };
    using std::integral_constant;
    auto by_nb = [&](auto sc) {
        switch (nb) {
            case 2: go(sc, integral_constant<int, 2>{}); break;
            case 4: go(sc, integral_constant<int, 4>{}); break;
            case 8: go(sc, integral_constant<int, 8>{}); break;
            default: go(sc, integral_constant<int, 16>{}); break;
        }
    };
    switch (S) {
        case 1: by_nb(integral_constant<int, 1>{}); break;
        case 2: by_nb(integral_constant<int, 2>{}); break;
        case 4:
            if (nb <= 8) {
                if (nb == 2) go(integral_constant<int, 4>{}, integral_constant<int, 2>{});
                else if (nb == 4) go(integral_constant<int, 4>{}, integral_constant<int, 4>{});
                else go(integral_constant<int, 4>{}, integral_constant<int, 8>{});
            }
            break;
        default: go(integral_constant<int, 8>{}, integral_constant<int, 2>{}); break;
    }
}

}  // namespace

void svrg_inner(cudaStream_t s, const void *X, lra_dtype dt, int64_t ldx, int64_t dpad, int p,
                float *W, const float *Wt, const float *M, const int32_t *idx, const float *cval,
                int64_t m, float eta, float lam, int batch, float cscale) {
    if (m <= 0) return;  // an empty step sequence leaves W unchanged
    if (batch < 1 || batch > 16 || (batch & (batch - 1)) != 0) {
        set_error("batch must be a power of two in [1, 16]");
        throw Error{LRA_EINVAL};
    }
    // a stored X scaled by sigma (FP16 storage) gives r sigma times the true r;
    // c_i / sigma^2 in the stochastic term keeps every step the true one
    const float etac = eta * cscale;
    if (dt == LRA_BF16)
        inner_dispatch<__nv_bfloat16>(s, X, ldx, dpad, p, W, Wt, M, idx, cval, m, batch, eta, lam, etac);
    else if (dt == LRA_F16)
        inner_dispatch<__half>(s, X, ldx, dpad, p, W, Wt, M, idx, cval, m, batch, eta, lam, etac);
    else
        inner_dispatch<float>(s, X, ldx, dpad, p, W, Wt, M, idx, cval, m, batch, eta, lam, etac);
}

}  // namespace lra
