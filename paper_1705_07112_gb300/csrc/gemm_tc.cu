// Blackwell (sm_103a) tensor-core GEMM with the fused CPA epilogue.
//
//   out(i,j) = epi( sum_k A(i,k) B(j,k) ),  A: M x K, B: N x K, both BF16
//   K-major in global memory, FP32 accumulation in tensor memory (TMEM).
//
// Structure (one CTA per SM, persistent over output tiles of 128 x BN):
//   warp 0      TMA producer: cp.async.bulk.tensor loads of A and B
//               K-slices (64 elements = one 128-byte swizzle row) into a
//               ring of shared-memory stages, completion on mbarriers; with
//               K a multiple of 64 the operands are viewed as 3-D
//               {64, rows, K/64} so one load brings several slices.
//   warp 1      MMA issuer: allocates TMEM, one elected thread issues
//               tcgen05.mma kind::f16 (M=128, N=BN, K=16) per 32-byte K step,
//               tcgen05.commit frees a stage / publishes an accumulator.
//   warps 2..5  epilogue: tcgen05.ld 32x32b (one accumulator row per thread),
//               fused  D = s_acc*acc + s_c*C + s_c2*C2 + diag,  H += c_k D,
//               BF16 hi/lo copies of D, while the MMA warp fills the other
//               accumulator.  Symmetric outputs: only tiles meeting the upper
//               triangle are computed; the FP32 arrays are read and written at
//               the mirrored position (j,i), which is coalesced when each lane
//               owns one row, and the values for (i,j) go through a per-warp
//               shared-memory transpose so those stores are coalesced too.
// Split precision (nsplit = 3) runs the K loop three times over
// (A_hi,B_hi), (A_hi,B_lo), (A_lo,B_hi) into the same accumulator.
// The recurrence runs all its steps in one cooperative launch with a grid
// barrier per step; when each CTA owns at most one tile, the tile's FP32
// state (Psi_{k-1}, Psi_{k-2}, H) stays in tensor memory between steps and
// only the BF16 operand copies of each Psi_k go through global memory.
//
// Every mbarrier wait is bounded (~2 s of clock); on expiry the CTA raises
// an error flag, stops issuing work, drains the TMA loads it started, frees
// its TMEM and returns.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <cstdio>
#include <cstring>
#include <type_traits>
#include <mutex>

#include "internal.h"
#include "tc_ptx.h"

namespace cpa {
namespace {

using namespace tc;

constexpr int BM = 128;
constexpr int BK = 64;            // bf16 elements per 128-byte swizzle row
constexpr int kThreads = 192;
constexpr long long kWaitCycles = 4000000000LL;   // ~2 s at 2 GHz

__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, uint64_t *bar, int x, int y) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::"r"(
            su32(dst)),
        "l"(map), "r"(su32(bar)), "r"(x), "r"(y)
        : "memory");
}
// 3-D load (x, y, z): used for operand maps viewed as {64, rows, K/64}, so
// one instruction brings several consecutive 128-byte K slices.
__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, uint64_t *bar, int x, int y, int z) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5}], [%2];" ::"r"(
            su32(dst)),
        "l"(map), "r"(su32(bar)), "r"(x), "r"(y), "r"(z)
        : "memory");
}

__device__ __forceinline__ void tma_store_2d(const CUtensorMap *map, const void *src, int x, int y) {
    asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%2, %3}], [%1];" ::"l"(map),
                 "r"(su32(src)), "r"(x), "r"(y)
                 : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read_all() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

// Operand maps of the main loop and the 32 x 32 block maps of the epilogue
// (FP32 C, C2, H, D and BF16 hi/lo copies of D).
// Per ring parity of the recurrence (a single product uses parity 0): the B
// operand and the epilogue block maps (C = D updated in place, C2, D hi/lo).
struct StepMaps {
    CUtensorMap b_hi, b_lo;
    CUtensorMap c, c2, d, dhi, dlo;
};
struct TileMaps {
    CUtensorMap a_hi, a_lo, h;
    StepMaps s[2];
};

// Several recurrence steps in one cooperative launch.  Step k uses ring slot
// k & 1: D = C = z[k&1] (Psi_{k-2} overwritten by Psi_k), C2 = z[(k&1)^1]
// (Psi_{k-1}), BF16 copies zhi/zlo[k&1], B operand zhi/zlo[(k&1)^1]; step 2
// has no C and subtracts Id on the diagonal.  A grid barrier (counter *bar,
// zeroed before the launch) separates the steps.
struct MultiStep {
    int multi = 0;
    int k_first = 0, k_end = 1;
    float *z[2] = {nullptr, nullptr};
    __nv_bfloat16 *zhi[2] = {nullptr, nullptr}, *zlo[2] = {nullptr, nullptr};
    unsigned int *bar = nullptr;
    // Clenshaw's sum instead of the forward recurrence: step k produces
    // b_{L-1-k} = 2 B_hat b_{L-k} - b_{L+1-k} + c_{L-1-k} Id in the same ring
    // (b_{L-1} = c_{L-1} Id enters the first step as a diagonal term), no
    // running sum; the last step writes b_0 into H's array
    int clenshaw = 0;
    int L = 0;
    // resident: every CTA owns at most one tile, whose FP32 Psi_{k-1},
    // Psi_{k-2} and H (forward sum) stay in tensor memory between steps
    // (columns 2 BN.. after the two accumulators); only the first step reads
    // them from global memory and only the last writes H back (Clenshaw: the
    // last step also applies the closing H = (b_0 - b_2) / 2).  The FP32
    // ring arrays are then not written during the launch.
    int resident = 0;
    // grid-barrier wait limit in clock cycles; stall: the first barrier
    // expects one arrival more than the grid makes (tests of the timeout
    // path: it then ends only by the limit, every CTA stops after its step)
    long long wait_cycles = kDefaultWaitCycles;
    int stall = 0;
    // number of terms chosen on the device (learned order): the launch runs
    // the steps k_first <= k < min(k_end, *L_dev); null: k_end as given
    const int *L_dev = nullptr;
    // occupancy of the A operand (the thresholded At of the sparsity-based
    // reduction): amask[tm * mask_groups + zg] = 0 when rows tm*128.. of A
    // are zero over the zg-th group of K slices loaded per stage; such
    // groups are neither loaded nor multiplied (their products are exact
    // zeros), except group 0, which starts each accumulator
    const uint8_t *amask = nullptr;
    int mask_groups = 0;
};

// Occupancy of A in tiles of 128 rows x (width) columns: one block per tile,
// any nonzero hi or lo part marks it.
__global__ void amask_kernel(const __nv_bfloat16 *__restrict__ hi, const __nv_bfloat16 *__restrict__ lo, int64_t ld,
                             int rows, int K, int width, uint8_t *mask, int groups) {
    const int tm = blockIdx.y, zg = blockIdx.x;
    int any = 0;
    for (int e = threadIdx.x; e < 128 * width; e += blockDim.x) {
        const int r = tm * 128 + e / width, c = zg * width + e % width;
        if (r < rows && c < K) {
            const int64_t o = (int64_t)r * ld + c;
            if (__bfloat16_as_ushort(hi[o]) & 0x7FFF) any = 1;
            if (lo && (__bfloat16_as_ushort(lo[o]) & 0x7FFF)) any = 1;
        }
    }
    any = __syncthreads_or(any);
    if (threadIdx.x == 0) mask[tm * groups + zg] = any ? 1 : 0;
}

__device__ __forceinline__ void fence_proxy_async_global() {
    asm volatile("fence.proxy.async.global;" ::: "memory");
}

// Shared memory of one epilogue warp: three FP32 32 x 32 blocks (C -> D in
// place, C2, H in place), two BF16 32 x 32 blocks (hi/lo copies of D at the
// mirrored position) and a padded 32 x 33 word transpose buffer.
struct EpiSmem {
    float c[32 * 32];
    float c2[32 * 32];
    float h[32 * 32];
    __nv_bfloat16 hi[32 * 32];
    __nv_bfloat16 lo[32 * 32];
    uint32_t t[32 * 33];
    uint32_t pad[32 - (32 * 33) % 32];
};

// A stage holds up to kG consecutive 64-element K slices of A and of B,
// stored slice after slice (each slice a 128-byte swizzled tile), so one
// 3-D TMA instruction per operand fills it: issuing TMA instructions costs
// about 100 cycles each, which bounds a tile's main loop when every K slice
// takes its own pair of instructions.
template <int BN>
struct Smem {
    static constexpr int kG = (BN == 256) ? 1 : 2;
    static constexpr int kStageA = BM * BK * 2 * kG;
    static constexpr int kStageB = BN * BK * 2 * kG;
    static constexpr int kStages = (BN == 128) ? 2 : 3;   // 256: 3 x 48 KB, 128: 2 x 64, 64: 3 x 48, 32: 3 x 40
    static constexpr int kBytes =
        kStages * (kStageA + kStageB) + 4 * (int)sizeof(EpiSmem) + 1024 /* align */ + 256 /* barriers */;
};

// ------------------------------------------------------------------ epilogue

__device__ __forceinline__ uint32_t pack_hilo(float v) {
    __nv_bfloat16 hi = __float2bfloat16_rn(v);
    __nv_bfloat16 lo = __float2bfloat16_rn(v - __bfloat162float(hi));
    return (uint32_t)__bfloat16_as_ushort(hi) | ((uint32_t)__bfloat16_as_ushort(lo) << 16);
}

// Writes the 32 x 32 block held in the transpose buffer (word [r][c] is
// element (r0 + r, j0 + c)) to row-major global memory with coalesced
// stores; `upper` keeps only c0 + c > r0 + r.  mode 0: FP32 to D,
// mode 1: BF16 hi (low half) / lo (high half) to Dhi / Dlo.
__device__ __forceinline__ void store_transposed(const Epilogue &e, const uint32_t *t, int mode, int M, int N, int r0,
                                                 int j0, int lane, bool upper) {
    const int jj = j0 + lane;
    if (jj >= N) return;
#pragma unroll 8
    for (int rr = 0; rr < 32; ++rr) {
        const int ii = r0 + rr;
        if (ii >= M || (upper && jj <= ii)) continue;
        const uint32_t val = t[rr * 33 + lane];
        if (mode == 0) {
            e.D[(int64_t)ii * e.ldd + jj] = __uint_as_float(val);
        } else {
            e.Dhi[(int64_t)ii * e.ldb + jj] = __ushort_as_bfloat16((unsigned short)(val & 0xFFFF));
            if (e.Dlo) e.Dlo[(int64_t)ii * e.ldb + jj] = __ushort_as_bfloat16((unsigned short)(val >> 16));
        }
    }
}

// BF16 hi/lo parts of the 32 x 32 block held in the transpose buffer (word
// [r][c] is element (r0 + r, j0 + c), hi in the low half) to Dhi / Dlo with
// 16-byte stores: lane l writes columns 8 (l % 4) .. +7 of rows l / 4 + 8 s,
// s = 0..3 (conflict-free reads of the buffer); a partial row at the right
// edge falls back to 2-byte stores.
__device__ __forceinline__ void store_transposed_bf16x8(const Epilogue &e, const uint32_t *t, int M, int N, int r0,
                                                        int j0, int lane) {
    const int q = lane & 3, cc = 8 * q, jj = j0 + cc;
#pragma unroll
    for (int sp = 0; sp < 4; ++sp) {
        const int rr = (lane >> 2) + 8 * sp, ii = r0 + rr;
        if (ii >= M || jj >= N) continue;
        uint32_t w[8];
#pragma unroll
        for (int x = 0; x < 8; ++x) w[x] = t[rr * 33 + cc + x];
        const int64_t o = (int64_t)ii * e.ldb + jj;
        if (jj + 8 <= N) {
            uint4 h4, l4;
            h4.x = (w[0] & 0xFFFFu) | (w[1] << 16);
            h4.y = (w[2] & 0xFFFFu) | (w[3] << 16);
            h4.z = (w[4] & 0xFFFFu) | (w[5] << 16);
            h4.w = (w[6] & 0xFFFFu) | (w[7] << 16);
            *reinterpret_cast<uint4 *>(e.Dhi + o) = h4;
            if (e.Dlo) {
                l4.x = (w[0] >> 16) | (w[1] & 0xFFFF0000u);
                l4.y = (w[2] >> 16) | (w[3] & 0xFFFF0000u);
                l4.z = (w[4] >> 16) | (w[5] & 0xFFFF0000u);
                l4.w = (w[6] >> 16) | (w[7] & 0xFFFF0000u);
                *reinterpret_cast<uint4 *>(e.Dlo + o) = l4;
            }
        } else {
            for (int x = 0; x < 8 && jj + x < N; ++x) {
                e.Dhi[o + x] = __ushort_as_bfloat16((unsigned short)(w[x] & 0xFFFF));
                if (e.Dlo) e.Dlo[o + x] = __ushort_as_bfloat16((unsigned short)(w[x] >> 16));
            }
        }
    }
}

// Symmetric output, one 32 x 32 block of the accumulator held by a warp:
// lane l owns row i = r0 + l, acc[c] is column j = j0 + c, j0 >= r0.
// The FP32 arrays live in the lower triangle, so the block is handled at
// its mirrored position (rows j0.., columns r0..), moved by TMA:
//   loads C, C2, H -> es.c, es.c2, es.h  ([j - j0][i - r0]),
//   v = s_acc acc + s_c C + s_c2 C2 + diag,  es.c = v,  es.h += c_k v,
//   es.hi/lo = BF16 parts of v,  TMA stores of D, H, Dhi, Dlo;
// the BF16 parts for the upper positions (i, j) go out through the
// transpose buffer.  A diagonal block (j0 == r0) is written in full at its
// own position, each pair (i,j), (j,i) taking the value of the upper
// element.  Only lane 0 issues TMA operations.
// Issues the TMA loads of one block's inputs (C, C2, H at the mirrored
// position) into the warp's buffers, once the previous block's TMA stores
// have finished reading them.
// Returns whether loads were issued (a phase of `bar` is then pending).
__device__ __forceinline__ bool epilogue_issue_loads(const Epilogue &e, const StepMaps &maps, const CUtensorMap &hmap,
                                                     int r0, int j0, int lane, EpiSmem &es, uint64_t *bar) {
    fence_proxy_async();
    __syncwarp();
    const bool any = e.C || e.C2 || e.H;
    if (lane == 0) {
        bulk_wait_read_all();
        if (any) {
            const uint32_t bytes = 4096u * ((e.C ? 1u : 0u) + (e.C2 ? 1u : 0u) + (e.H ? 1u : 0u));
            mbar_expect_tx(bar, bytes);
            if (e.C) tma_load_2d(es.c, &maps.c, bar, r0, j0);
            if (e.C2) tma_load_2d(es.c2, &maps.c2, bar, r0, j0);
            if (e.H) tma_load_2d(es.h, &hmap, bar, r0, j0);
        }
    }
    __syncwarp();
    return any;
}

__device__ __forceinline__ void epilogue_sym_block(const Epilogue &e, const StepMaps &maps, const CUtensorMap &hmap,
                                                   float ck, int M, int N,
                                                   int r0, int j0, int lane, const float *acc, EpiSmem &es,
                                                   uint64_t *bar, uint32_t &phase, volatile int *abort_flag,
                                                   bool preloaded, const CUtensorMap *dmap, int next_j0, bool &epend) {
    const bool diag = (j0 == r0);
    const bool any_load = e.C || e.C2 || e.H;
    if (!preloaded) epend = epilogue_issue_loads(e, maps, hmap, r0, j0, lane, es, bar) || epend;
    if (any_load) {
        if (mbar_wait(bar, phase, abort_flag)) epend = false;
        phase ^= 1u;
    }
    const int i = r0 + lane;
    uint32_t hl[32];
    if (!diag) {
        // the inputs' scales, zero where an input is absent (its buffer is
        // then not read); groups of 8 columns issue all their shared-memory
        // loads before their stores, so the loads overlap
        const float sa = e.s_acc, sc = e.C ? e.s_c : 0.f, sc2 = e.C2 ? e.s_c2 : 0.f;
        const bool hasc = e.C != nullptr, hasc2 = e.C2 != nullptr, hash = e.H != nullptr;
#pragma unroll
        for (int g = 0; g < 32; g += 8) {
            float cv[8], c2v[8], hv[8];
#pragma unroll
            for (int x = 0; x < 8; ++x) {
                cv[x] = hasc ? es.c[(g + x) * 32 + lane] : 0.f;
                c2v[x] = hasc2 ? es.c2[(g + x) * 32 + lane] : 0.f;
                hv[x] = hash ? es.h[(g + x) * 32 + lane] : 0.f;
            }
#pragma unroll
            for (int x = 0; x < 8; ++x) {
                const int c = g + x;
                const float v = fmaf(sc2, c2v[x], fmaf(sc, cv[x], sa * acc[c]));
                es.c[c * 32 + lane] = v;
                if (hash) es.h[c * 32 + lane] = fmaf(ck, v, hv[x]);
                const uint32_t p = pack_hilo(v);
                hl[c] = p;
                es.hi[c * 32 + lane] = __ushort_as_bfloat16((unsigned short)(p & 0xFFFF));
                es.lo[c * 32 + lane] = __ushort_as_bfloat16((unsigned short)(p >> 16));
            }
        }
    } else {
        // read every input first: the stores below touch both triangles
        float cv[32], c2v[32], hv[32];
#pragma unroll
        for (int c = 0; c < 32; ++c) {
            const int a = c >= lane ? c * 32 + lane : lane * 32 + c;   // lower-triangle copy
            cv[c] = e.C ? es.c[a] : 0.f;
            c2v[c] = e.C2 ? es.c2[a] : 0.f;
            hv[c] = e.H ? es.h[a] : 0.f;
        }
        __syncwarp();
#pragma unroll
        for (int c = 0; c < 32; ++c) {
            if (c < lane) continue;   // the pair is written by lane c
            float v = fmaf(e.s_c2, c2v[c], fmaf(e.s_c, cv[c], e.s_acc * acc[c]));
            if (c == lane) v += e.diag;
            const float hn = fmaf(ck, v, hv[c]);
            const uint32_t p = pack_hilo(v);
            const __nv_bfloat16 bh = __ushort_as_bfloat16((unsigned short)(p & 0xFFFF));
            const __nv_bfloat16 bl = __ushort_as_bfloat16((unsigned short)(p >> 16));
            es.c[c * 32 + lane] = v;
            es.c[lane * 32 + c] = v;
            if (e.H) {
                es.h[c * 32 + lane] = hn;
                es.h[lane * 32 + c] = hn;
            }
            es.hi[c * 32 + lane] = bh;
            es.hi[lane * 32 + c] = bh;
            es.lo[c * 32 + lane] = bl;
            es.lo[lane * 32 + c] = bl;
        }
    }
    (void)i;
    fence_proxy_async();
    __syncwarp();
    if (lane == 0) {
        tma_store_2d(dmap, es.c, r0, j0);
        if (e.H) tma_store_2d(&hmap, es.h, r0, j0);
        if (e.Dhi) {
            tma_store_2d(&maps.dhi, es.hi, r0, j0);
            if (e.Dlo) tma_store_2d(&maps.dlo, es.lo, r0, j0);
        }
        bulk_commit();
    }
    // the next block's inputs do not depend on its accumulator: once this
    // block's inputs are no longer read (the stores above read c and h from
    // shared memory; the full-D copy below reads c), load them, so that
    // their latency overlaps this block's remaining stores and the next
    // block's accumulator read
    if (diag) {
        if (next_j0 >= 0) epend = epilogue_issue_loads(e, maps, hmap, r0, next_j0, lane, es, bar) || epend;
        return;
    }
    // upper positions (i, j): the transposed values of the mirrored block
    if (e.sym_full_d) {
#pragma unroll
        for (int c = 0; c < 32; ++c) es.t[lane * 33 + c] = __float_as_uint(es.c[c * 32 + lane]);
        __syncwarp();
        store_transposed(e, es.t, 0, M, N, r0, j0, lane, false);
        __syncwarp();
    }
    if (next_j0 >= 0) epend = epilogue_issue_loads(e, maps, hmap, r0, next_j0, lane, es, bar) || epend;
    if (e.Dhi) {
#pragma unroll
        for (int c = 0; c < 32; ++c) es.t[lane * 33 + c] = hl[c];
        __syncwarp();
        store_transposed_bf16x8(e, es.t, M, N, r0, j0, lane);
        __syncwarp();
    }
}

// Resident recurrence step, one 32 x 32 block of the accumulator held by a
// warp (lane l owns row r0 + l, acc[c] is column j0 + c, j0 >= r0).  The
// block's state lives in tensor memory in the same orientation: tC (Psi_{k-2},
// overwritten by Psi_k), tC2 (Psi_{k-1}) and tH (H, forward sum only), each
// the address of the block's first column in this warp's lane quarter.
// from_tmem = false (first step): the inputs come from global memory through
// the TMA block loads, as in the non-resident step.  The BF16 copies of
// Psi_k are written as in the non-resident step; FP32 D and H go to global
// memory only when store_d / store_h.  close: Clenshaw's last step, the
// value kept is (b_0 - b_2) / 2 with b_2 = C (+ close_diag on the diagonal
// when b_2 = c_{L-1} Id enters this same step).
__device__ __forceinline__ void epilogue_res_block(const Epilogue &e, const StepMaps &maps, const CUtensorMap &hmap,
                                                   float ck, int M, int N, int r0, int j0, int lane,
                                                   const float *acc, EpiSmem &es, uint64_t *bar, uint32_t &phase,
                                                   volatile int *abort_flag, bool preloaded, const CUtensorMap *dmap,
                                                   bool from_tmem, uint32_t tC, uint32_t tC2, uint32_t tH,
                                                   bool store_d, bool store_h, bool close, float close_diag,
                                                   bool &epend) {
    const bool diag = (j0 == r0);
    const bool hasc = e.C != nullptr, hasc2 = e.C2 != nullptr, hact = e.H != nullptr;
    if (from_tmem) {
        // the warp's buffers are rewritten below: the previous block's TMA
        // stores must have finished reading them
        if (lane == 0) bulk_wait_read_all();
        __syncwarp();
    } else {
        if (!preloaded) epend = epilogue_issue_loads(e, maps, hmap, r0, j0, lane, es, bar) || epend;
        if (hasc || hasc2 || hact) {
            if (mbar_wait(bar, phase, abort_flag)) epend = false;
            phase ^= 1u;
        }
    }
    uint32_t hl[32];
    if (!diag) {
        const float sa = e.s_acc, sc = hasc ? e.s_c : 0.f, sc2 = hasc2 ? e.s_c2 : 0.f;
#pragma unroll
        for (int g = 0; g < 32; g += 8) {
            float cv[8], c2v[8], hv[8];
            if (from_tmem) {
                tmem_ld8x3(tC + g, tC2 + g, tH + g, cv, c2v, hv);
#pragma unroll
                for (int x = 0; x < 8; ++x) {
                    cv[x] = hasc ? cv[x] : 0.f;
                    c2v[x] = hasc2 ? c2v[x] : 0.f;
                    hv[x] = hact ? hv[x] : 0.f;
                }
            } else {
#pragma unroll
                for (int x = 0; x < 8; ++x) {
                    cv[x] = hasc ? es.c[(g + x) * 32 + lane] : 0.f;
                    c2v[x] = hasc2 ? es.c2[(g + x) * 32 + lane] : 0.f;
                    hv[x] = hact ? es.h[(g + x) * 32 + lane] : 0.f;
                }
            }
            float vo[8], ho[8];
#pragma unroll
            for (int x = 0; x < 8; ++x) {
                const int c = g + x;
                float v = fmaf(sc2, c2v[x], fmaf(sc, cv[x], sa * acc[c]));
                if (close) v = 0.5f * (v - cv[x]);
                vo[x] = v;
                ho[x] = fmaf(ck, v, hv[x]);
                if (store_d) es.c[c * 32 + lane] = v;
                if (store_h) es.h[c * 32 + lane] = ho[x];
                const uint32_t p = pack_hilo(v);
                hl[c] = p;
                es.hi[c * 32 + lane] = __ushort_as_bfloat16((unsigned short)(p & 0xFFFF));
                es.lo[c * 32 + lane] = __ushort_as_bfloat16((unsigned short)(p >> 16));
            }
            tmem_st8(tC + g, vo);
            if (hact) tmem_st8(tH + g, ho);
            if (!from_tmem) tmem_st8(tC2 + g, c2v);   // Psi_{k-1} for the next step
        }
    } else {
        float cv[32], c2v[32], hv[32];
        if (from_tmem) {
            // the state holds both triangles of a diagonal block
            tmem_ld32(tC, cv);
            tmem_ld32(tC2, c2v);
            tmem_ld32(tH, hv);
#pragma unroll
            for (int c = 0; c < 32; ++c) {
                cv[c] = hasc ? cv[c] : 0.f;
                c2v[c] = hasc2 ? c2v[c] : 0.f;
                hv[c] = hact ? hv[c] : 0.f;
            }
        } else {
#pragma unroll
            for (int c = 0; c < 32; ++c) {
                const int a = c >= lane ? c * 32 + lane : lane * 32 + c;   // lower-triangle copy
                cv[c] = hasc ? es.c[a] : 0.f;
                c2v[c] = hasc2 ? es.c2[a] : 0.f;
                hv[c] = hact ? es.h[a] : 0.f;
            }
        }
        __syncwarp();
        const float diagv = epilogue_diag(e);
#pragma unroll
        for (int c = 0; c < 32; ++c) {
            if (c < lane) continue;   // the pair is written by lane c
            float v = fmaf(e.s_c2, c2v[c], fmaf(e.s_c, cv[c], e.s_acc * acc[c]));
            if (c == lane) v += diagv;
            if (close) v = 0.5f * (v - cv[c] - (c == lane ? close_diag : 0.f));
            const float hn = fmaf(ck, v, hv[c]);
            const uint32_t p = pack_hilo(v);
            const __nv_bfloat16 bh = __ushort_as_bfloat16((unsigned short)(p & 0xFFFF));
            const __nv_bfloat16 bl = __ushort_as_bfloat16((unsigned short)(p >> 16));
            es.c[c * 32 + lane] = v;
            es.c[lane * 32 + c] = v;
            if (hact) {
                es.h[c * 32 + lane] = hn;
                es.h[lane * 32 + c] = hn;
            }
            es.hi[c * 32 + lane] = bh;
            es.hi[lane * 32 + c] = bh;
            es.lo[c * 32 + lane] = bl;
            es.lo[lane * 32 + c] = bl;
        }
        __syncwarp();
        // this lane's row of the block (both triangles) into tensor memory
        if (!from_tmem) {
#pragma unroll
            for (int g = 0; g < 32; g += 8) tmem_st8(tC2 + g, c2v + g);   // Psi_{k-1} for the next step
        }
#pragma unroll
        for (int c = 0; c < 32; ++c) cv[c] = es.c[c * 32 + lane];
#pragma unroll
        for (int g = 0; g < 32; g += 8) tmem_st8(tC + g, cv + g);
        if (hact) {
#pragma unroll
            for (int c = 0; c < 32; ++c) hv[c] = es.h[c * 32 + lane];
#pragma unroll
            for (int g = 0; g < 32; g += 8) tmem_st8(tH + g, hv + g);
        }
    }
    tmem_st_wait();
    fence_proxy_async();
    __syncwarp();
    if (lane == 0) {
        if (store_d) tma_store_2d(dmap, es.c, r0, j0);
        if (store_h) tma_store_2d(&hmap, es.h, r0, j0);
        if (e.Dhi) {
            tma_store_2d(&maps.dhi, es.hi, r0, j0);
            if (e.Dlo) tma_store_2d(&maps.dlo, es.lo, r0, j0);
        }
        bulk_commit();
    }
    if (diag) return;
    if (e.Dhi) {
#pragma unroll
        for (int c = 0; c < 32; ++c) es.t[lane * 33 + c] = hl[c];
        __syncwarp();
        store_transposed_bf16x8(e, es.t, M, N, r0, j0, lane);
        __syncwarp();
    }
}

// General (non-symmetric) output: D(i,j) = s_acc acc + diag, stored through
// the transpose buffer.
__device__ __forceinline__ void epilogue_general_block(const Epilogue &e, int M, int N, int r0, int j0, int lane,
                                                       const float *acc, EpiSmem &es) {
    const int i = r0 + lane;
#pragma unroll
    for (int c = 0; c < 32; ++c) {
        float v = e.s_acc * acc[c];
        if (i == j0 + c) v += e.diag;
        es.t[lane * 33 + c] = __float_as_uint(v);
    }
    __syncwarp();
    store_transposed(e, es.t, 0, M, N, r0, j0, lane, false);
    __syncwarp();
}

// Output tile t of the persistent schedule.  Symmetric outputs visit only
// tiles meeting the upper triangle: in tile row tm these start at column
// tile (tm*BM)/BN.
__device__ __forceinline__ void tile_of(int t, int tiles_m, int tiles_n, int sym, int bn, int &tm, int &tn) {
    if (!sym) {
        tm = t / tiles_n;
        tn = t % tiles_n;
        return;
    }
    for (tm = 0; tm < tiles_m; ++tm) {
        const int first = (tm * BM) / bn;
        const int cnt = tiles_n - first;
        if (t < cnt) {
            tn = first + t;
            return;
        }
        t -= cnt;
    }
    tn = 0;
}

__host__ __device__ inline int count_tiles(int tiles_m, int tiles_n, int sym, int bn) {
    if (!sym) return tiles_m * tiles_n;
    int c = 0;
    for (int tm = 0; tm < tiles_m; ++tm) {
        int first = (tm * BM) / bn;
        if (first < tiles_n) c += tiles_n - first;
    }
    return c;
}

template <int BN>
__global__ void __launch_bounds__(kThreads, 1)
    gemm_tc_kernel(const __grid_constant__ TileMaps maps, int M, int N, int K, int nsplit, int g, Epilogue e,
                   MultiStep ms, int *err) {
    using S = Smem<BN>;
    constexpr int kStages = S::kStages;
    // two accumulators, plus three BN-column state slots when resident
    const uint32_t tmem_cols = ms.resident ? (BN == 32 ? 256u : 512u) : 2u * BN;
    constexpr uint32_t kIdesc = idesc_bf16(BM, BN);

    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t *sA = smem;
    uint8_t *sB = smem + kStages * S::kStageA;
    EpiSmem *epi = reinterpret_cast<EpiSmem *>(sB + kStages * S::kStageB);   // [4]
    uint64_t *bars = reinterpret_cast<uint64_t *>(epi + 4);
    uint64_t *full = bars;                 // [kStages]
    uint64_t *empty = bars + kStages;      // [kStages]
    uint64_t *tfull = bars + 2 * kStages;  // [2]
    uint64_t *tempty = tfull + 2;          // [2]
    uint64_t *ebar = tempty + 2;           // [4] epilogue TMA loads
    uint64_t *stepbar = ebar + 4;          // next step may load (multi-step)
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(stepbar + 1);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int tiles_m = (M + BM - 1) / BM, tiles_n = (N + BN - 1) / BN;
    // last step + 1 (the terms of a learned order are read from the device)
    const int k_end = ms.L_dev ? max(ms.k_first, min(ms.k_end, __ldg(ms.L_dev))) : ms.k_end;
    const int sym = e.symmetric_upper;
    const int ntiles = count_tiles(tiles_m, tiles_n, sym, BN);
    const int kb_per = (K + BK - 1) / BK;
    // g > 0: 3-D operand maps with g slices per load (g divides kb_per);
    // g == 0: 2-D maps, one slice per stage; g < 0 (split products, two
    // slots per stage): 2-D maps, a stage holds one K slice of A hi, A lo,
    // B hi and B lo and takes all three split products (hi*hi, hi*lo, lo*hi)
    // from it, so each operand slice is fetched once instead of twice
    const bool inter = g < 0 && S::kG == 2 && nsplit == 3;
    const int nkb = inter ? kb_per : kb_per * nsplit;
    const bool tma3d = S::kG > 1 && g > 0;
    const int gs = tma3d ? g : 1;
    const uint32_t stage_bytes = (uint32_t)(inter ? 2 : gs) * (uint32_t)(BM + BN) * (uint32_t)(BK * 2);

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&tfull[b], 1);
            mbar_init(&tempty[b], 4);
        }
        for (int q = 0; q < 4; ++q) mbar_init(&ebar[q], 1);
        mbar_init(stepbar, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tmem_slot)),
                     "r"(tmem_cols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem_base = *tmem_slot;

    if (warp == 0) {
        // ------------------------------------------------------------ producer
        if (lane == 0) {
            int stage = 0;
            uint32_t phase = 0, sphase = 0;
            uint32_t armed_mask = 0, armed_phase = 0;   // per stage: armed at least once / phase it was armed in
            for (int k = ms.k_first; k < k_end && !*abort_flag; ++k) {
                if (ms.multi && k > ms.k_first) {
                    // the previous step's outputs are complete in every CTA
                    if (!mbar_wait(stepbar, sphase, abort_flag)) break;
                    sphase ^= 1;
                    fence_proxy_async_global();
                }
                const StepMaps &sm = maps.s[ms.multi ? (k & 1) : 0];
                for (int t = blockIdx.x; t < ntiles && !*abort_flag; t += gridDim.x) {
                    int tm, tn;
                    tile_of(t, tiles_m, tiles_n, sym, BN, tm, tn);
                    const int m0 = tm * BM, n0 = tn * BN;
                    for (int kb = 0; kb < nkb; kb += gs) {
                        const int seg = inter ? 0 : kb / kb_per, z = inter ? kb : kb % kb_per;
                        if (ms.amask && z > 0 && !ms.amask[tm * ms.mask_groups + z / gs]) continue;
                        if (!mbar_wait(&empty[stage], phase ^ 1, abort_flag)) break;
                        const CUtensorMap *ma = (seg < 2) ? &maps.a_hi : &maps.a_lo;
                        const CUtensorMap *mb = (seg == 1) ? &sm.b_lo : &sm.b_hi;
                        mbar_expect_tx(&full[stage], stage_bytes);
                        if (inter) {
                            // slot 1 starts BM (BN) 128-byte rows after slot 0
                            uint8_t *a0 = sA + stage * S::kStageA, *b0 = sB + stage * S::kStageB;
                            tma_load_2d(a0, &maps.a_hi, &full[stage], z * BK, m0);
                            tma_load_2d(a0 + BM * BK * 2, &maps.a_lo, &full[stage], z * BK, m0);
                            tma_load_2d(b0, &sm.b_hi, &full[stage], z * BK, n0);
                            tma_load_2d(b0 + BN * BK * 2, &sm.b_lo, &full[stage], z * BK, n0);
                        } else if (tma3d) {
                            tma_load_3d(sA + stage * S::kStageA, ma, &full[stage], 0, m0, z);
                            tma_load_3d(sB + stage * S::kStageB, mb, &full[stage], 0, n0, z);
                        } else {
                            tma_load_2d(sA + stage * S::kStageA, ma, &full[stage], z * BK, m0);
                            tma_load_2d(sB + stage * S::kStageB, mb, &full[stage], z * BK, n0);
                        }
                        armed_mask |= 1u << stage;
                        armed_phase = (armed_phase & ~(1u << stage)) | (phase << stage);
                        if (++stage == kStages) {
                            stage = 0;
                            phase ^= 1;
                        }
                    }
                }
            }
            if (*abort_flag) {
                // drain: the last load armed on each stage completes the full
                // barrier phase it was armed in; wait for it (bounded) so no
                // copy is still writing shared memory when the CTA exits
                for (int s2 = 0; s2 < kStages; ++s2) {
                    if (!(armed_mask & (1u << s2))) continue;
                    const uint32_t ph = (armed_phase >> s2) & 1u;
                    long long t0 = clock64();
                    while (!mbar_try_wait(&full[s2], ph) && clock64() - t0 < kWaitCycles) {
                    }
                }
            }
        }
    } else if (warp == 1) {
        // ------------------------------------------------------------ MMA issuer
        if (lane == 0) {
            int stage = 0;
            uint32_t phase = 0;
            uint32_t tphase[2] = {0, 0};
            int local = 0;
            bool ok = true;
            for (int k = ms.k_first; k < k_end && ok && !*abort_flag; ++k) {
                for (int t = blockIdx.x; t < ntiles && !*abort_flag; t += gridDim.x, ++local) {
                    const int buf = local & 1;
                    if (!mbar_wait(&tempty[buf], tphase[buf] ^ 1, abort_flag)) {
                        ok = false;
                        break;
                    }
                    tphase[buf] ^= 1;
                    fence_after();
                    const uint32_t d_tmem = tmem_base + (uint32_t)(buf * BN);
                    int tmm = 0, tnn = 0;
                    if (ms.amask) tile_of(t, tiles_m, tiles_n, sym, BN, tmm, tnn);
                    for (int kb = 0; kb < nkb; kb += gs) {
                        if (ms.amask && (kb % kb_per) > 0 && !ms.amask[tmm * ms.mask_groups + (kb % kb_per) / gs])
                            continue;
                        if (!mbar_wait(&full[stage], phase, abort_flag)) {
                            ok = false;
                            break;
                        }
                        fence_after();
                        const uint64_t da = smem_desc(su32(sA + stage * S::kStageA));
                        const uint64_t db = smem_desc(su32(sB + stage * S::kStageB));
                        if (inter) {
                            // hi*hi, hi*lo, lo*hi of this K slice (slot 1 = lo)
                            const uint64_t dal = da + (uint64_t)(BM * 8), dbl = db + (uint64_t)(BN * 8);
#pragma unroll
                            for (int kk = 0; kk < BK / 16; ++kk) {
                                mma_bf16(d_tmem, da + 2 * kk, db + 2 * kk, kIdesc, (kb > 0 || kk > 0) ? 1u : 0u);
                                mma_bf16(d_tmem, da + 2 * kk, dbl + 2 * kk, kIdesc, 1u);
                                mma_bf16(d_tmem, dal + 2 * kk, db + 2 * kk, kIdesc, 1u);
                            }
                        }
                        for (int sub = 0; sub < (inter ? 0 : gs); ++sub) {
                            // slice sub starts BM (BN) 128-byte rows further on;
                            // descriptor addresses count 16-byte units
                            const uint64_t das = da + (uint64_t)(sub * BM * 8), dbs = db + (uint64_t)(sub * BN * 8);
#pragma unroll
                            for (int kk = 0; kk < BK / 16; ++kk)
                                mma_bf16(d_tmem, das + 2 * kk, dbs + 2 * kk, kIdesc,
                                         (kb > 0 || sub > 0 || kk > 0) ? 1u : 0u);
                        }
                        mma_commit(&empty[stage]);
                        if (++stage == kStages) {
                            stage = 0;
                            phase ^= 1;
                        }
                    }
                    if (!ok) break;
                    mma_commit(&tfull[buf]);
                }
            }
        }
    } else {
        // ------------------------------------------------------------ epilogue
        const int quarter = warp & 3;   // TMEM lanes 32*quarter .. +31
        EpiSmem &es = epi[quarter];
        uint64_t *bar = &ebar[quarter];
        uint32_t ephase = 0;
        bool epend = false;   // a phase of this warp's block-load barrier is still to complete
        uint32_t tphase[2] = {0, 0};
        int local = 0;
        unsigned int target = 0;
        bool alive = true;
        for (int k = ms.k_first; k < k_end && alive; ++k) {
            Epilogue es_e = e;
            const int par = ms.multi ? (k & 1) : 0;
            bool final_to_h = false;
            if (ms.multi && !ms.clenshaw) {
                es_e.D = ms.z[par];
                es_e.C = (k == 2) ? nullptr : ms.z[par];
                es_e.C2 = ms.z[par ^ 1];
                es_e.Dhi = ms.zhi[par];
                es_e.Dlo = ms.zlo[par];
                es_e.diag = (k == 2) ? -1.f : 0.f;
                es_e.k = k;
            } else if (ms.multi) {
                const int kk = ms.L - 1 - k;   // b_kk
                const bool first = (k == ms.k_first);
                final_to_h = (kk == 0);
                es_e.D = final_to_h ? e.H : ms.z[par];
                es_e.C = first ? nullptr : ms.z[par];   // b_{kk+2}
                es_e.C2 = ms.z[par ^ 1];                 // b_{kk+1}
                es_e.Dhi = ms.zhi[par];
                es_e.Dlo = ms.zlo[par];
                es_e.diag = (float)(e.coef[kk] - (first ? e.coef[ms.L - 1] : 0.0));
                es_e.H = nullptr;
                es_e.k = k;
            }
            const CUtensorMap *dmap = final_to_h ? &maps.h : &maps.s[par].d;
            const float ck = es_e.H ? (float)es_e.coef[es_e.k] : 0.f;
            // resident state: slot par takes Psi_k over Psi_{k-2}, slot par^1
            // holds Psi_{k-1}, then H
            const bool res = BN <= 64 && ms.multi && ms.resident;
            const bool first = (k == ms.k_first), last = (k + 1 == k_end);
            const uint32_t sC = (uint32_t)(2 * BN + par * BN), sC2 = (uint32_t)(2 * BN + (par ^ 1) * BN),
                           sH = (uint32_t)(4 * BN);
            const bool close = res && final_to_h;
            const float close_diag = (close && first) ? (float)e.coef[ms.L - 1] : 0.f;
            const bool store_h = res && last && es_e.H != nullptr;
            for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++local) {
                const int buf = local & 1;
                int tm, tn;
                tile_of(t, tiles_m, tiles_n, sym, BN, tm, tn);
                const int r0 = tm * BM + quarter * 32, n0 = tn * BN;
                // the first block's inputs do not depend on the accumulator:
                // load them while the MMAs of this tile are still running
                int c_pre = -1;
                if (sym && r0 < M && (!res || first)) {
                    for (int c = 0; c < BN / 32; ++c) {
                        const int j0 = n0 + c * 32;
                        if (j0 < N && j0 >= r0) {
                            c_pre = c;
                            break;
                        }
                    }
                    if (c_pre >= 0)
                        epend = epilogue_issue_loads(es_e, maps.s[par], maps.h, r0, n0 + c_pre * 32, lane, es, bar) ||
                                epend;
                }
                if (!mbar_wait(&tfull[buf], tphase[buf], abort_flag)) {
                    alive = false;
                    break;
                }
                tphase[buf] ^= 1;
                fence_after();
                const uint32_t trow = tmem_base + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(buf * BN);
#pragma unroll 1
                for (int c = 0; c < BN / 32; ++c) {
                    float acc[32];
                    tmem_ld32(trow + (uint32_t)(c * 32), acc);
                    const int j0 = n0 + c * 32;
                    if (r0 >= M || j0 >= N) continue;
                    if (sym) {
                        if (j0 < r0) continue;   // block below the diagonal: written as another block's mirror
                        if constexpr (BN <= 64) {
                          if (res) {
                            const uint32_t tq = tmem_base + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(c * 32);
                            epilogue_res_block(es_e, maps.s[par], maps.h, ck, M, N, r0, j0, lane, acc, es, bar,
                                               ephase, abort_flag, c == c_pre, dmap, !first, tq + sC, tq + sC2,
                                               tq + sH, final_to_h, store_h, close, close_diag, epend);
                            continue;
                          }
                        }
                        // the tile's next block on or above the diagonal: its
                        // inputs are loaded ahead, at the end of this block
                        int c_next = -1;
                        for (int c2 = c + 1; c2 < BN / 32; ++c2) {
                            const int jn = n0 + c2 * 32;
                            if (jn < N && jn >= r0) {
                                c_next = c2;
                                break;
                            }
                        }
                        epilogue_sym_block(es_e, maps.s[par], maps.h, ck, M, N, r0, j0, lane, acc, es, bar, ephase,
                                           abort_flag, c == c_pre, dmap, c_next >= 0 ? n0 + c_next * 32 : -1, epend);
                        if (c_next >= 0) c_pre = c_next;
                    } else {
                        epilogue_general_block(es_e, M, N, r0, j0, lane, acc, es);
                    }
                }
                fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&tempty[buf]);
            }
            if (ms.multi && k + 1 < k_end && alive) {
                // step k done in this CTA: stores complete and ordered for the
                // async proxy, then one grid-wide barrier, then the producer
                // may load step k+1's operands
                if (lane == 0) bulk_wait_all();
                __syncwarp();
                fence_proxy_async_global();
                __threadfence();
                asm volatile("bar.sync 1, 128;" ::: "memory");
                if (threadIdx.x == 64) {
                    target += gridDim.x + ((ms.stall && k == ms.k_first) ? 1u : 0u);
                    asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(ms.bar) : "memory");
                    const long long t0 = clock64();
                    while (true) {
                        unsigned int v;
                        asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(ms.bar) : "memory");
                        if (v >= target) break;
                        if (clock64() - t0 > ms.wait_cycles) {
                            *abort_flag = 1;
                            break;
                        }
                    }
                    fence_proxy_async_global();
                    mbar_arrive(stepbar);
                }
                asm volatile("bar.sync 1, 128;" ::: "memory");
                fence_proxy_async_global();
                if (*abort_flag) alive = false;
            }
        }
        // the last TMA stores must complete before the CTA exits, and a block
        // load still in flight (a wait that gave up) must land first
        if (lane == 0) {
            bulk_wait_all();
            if (epend) {
                const long long t0 = clock64();
                while (!mbar_try_wait(bar, ephase) && clock64() - t0 < kWaitCycles) {
                }
            }
        }
        __syncwarp();
    }

    fence_before();
    __syncthreads();
    if (warp == 1) {
        fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(tmem_cols)
                     : "memory");
    }
    if (threadIdx.x == 0 && *abort_flag) atomicExch(err, CPA_ERR_TIMEOUT);
}

// ------------------------------------------------------------------- host side

PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
std::once_flag g_encode_once;

bool load_encode() {
    std::call_once(g_encode_once, [] {
        cudaDriverEntryPointQueryResult q;
        void *fn = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    });
    return g_encode != nullptr;
}

// Operand map viewed as {64, rows, K/64} (K a multiple of 64): a box of g
// consecutive 128-byte swizzled K slices, each box_rows rows high, lands as g
// stacked slices in shared memory.
bool make_map3(CUtensorMap *map, const __nv_bfloat16 *ptr, int64_t ld, int rows, int K, int box_rows, int g) {
    cuuint64_t dims[3] = {(cuuint64_t)BK, (cuuint64_t)rows, (cuuint64_t)(K / BK)};
    cuuint64_t strides[2] = {(cuuint64_t)(ld * 2), (cuuint64_t)(BK * 2)};
    cuuint32_t box[3] = {(cuuint32_t)BK, (cuuint32_t)box_rows, (cuuint32_t)g};
    cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = g_encode(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, (void *)ptr, dims, strides, box, estr,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

// Operand map: BF16 rows of K elements, 128-byte swizzled K slices.
bool make_map(CUtensorMap *map, const __nv_bfloat16 *ptr, int64_t ld, int rows, int K, int box_rows) {
    cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)(ld * 2)};
    cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = g_encode(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, (void *)ptr, dims, strides, box, estr,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

// Epilogue block map: 32 x 32 elements of a rows x cols row-major array.
bool make_block_map(CUtensorMap *map, const void *ptr, CUtensorMapDataType type, int esize, int64_t ld, int rows,
                    int cols) {
    cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)(ld * esize)};
    cuuint32_t box[2] = {32, 32};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = g_encode(map, type, 2, (void *)ptr, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                          CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

// Fallback error word of each device, for calls that pass none (one word
// per device: a kernel must never be handed another GPU's memory).
constexpr int kMaxDevices = 64;
int *g_err_dev[kMaxDevices] = {};
std::mutex g_err_mu;

cudaError_t device_err_word(int **out) {
    int dev = 0;
    cudaError_t r = cudaGetDevice(&dev);
    if (r != cudaSuccess) return r;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_err_mu);
    if (!g_err_dev[dev]) {
        int *p = nullptr;
        r = cudaMalloc(&p, sizeof(int));
        if (r != cudaSuccess) return r;
        r = cudaMemset(p, 0, sizeof(int));
        if (r != cudaSuccess) {
            cudaFree(p);
            return r;
        }
        g_err_dev[dev] = p;
    }
    *out = g_err_dev[dev];
    return cudaSuccess;
}

template <int BN>
cudaError_t launch(int M, int N, int K, const TcOperand &A, const TcOperand &B, int nsplit, const Epilogue &e,
                   const MultiStep &ms, cudaStream_t st, int num_sms) {
    using S = Smem<BN>;
    cudaError_t ra = ensure_smem_limit((const void *)gemm_tc_kernel<BN>, S::kBytes);
    if (ra != cudaSuccess) return ra;
    int *err = e.err;
    if (!err) {
        ra = device_err_word(&err);
        if (ra != cudaSuccess) return ra;
    }
    TileMaps maps;
    memset(&maps, 0, sizeof(maps));
    const CUtensorMapDataType f32 = CU_TENSOR_MAP_DATA_TYPE_FLOAT32, b16 = CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
    const __nv_bfloat16 *alo = A.lo ? A.lo : A.hi;
    // split products with two-slot stages: interleaved hi/lo slices (2-D
    // maps, g = -1); else grouped 3-D loads, which need whole 64-element
    // slices (no K tail to fill)
    const int g = (S::kG == 2 && nsplit == 3) ? -1
                  : (S::kG > 1 && K % BK == 0 && (K / BK) % S::kG == 0) ? S::kG : 0;
    auto opmap = [&](CUtensorMap *m, const __nv_bfloat16 *ptr, int64_t ld, int rows, int box_rows) {
        return g > 0 ? make_map3(m, ptr, ld, rows, K, box_rows, g) : make_map(m, ptr, ld, rows, K, box_rows);
    };
    if (!opmap(&maps.a_hi, A.hi, A.ld, A.rows, BM) || !opmap(&maps.a_lo, alo, A.ld, A.rows, BM))
        return cudaErrorInvalidValue;
    if (e.H && !make_block_map(&maps.h, e.H, f32, 4, e.ldh, M, N)) return cudaErrorInvalidValue;
    for (int par = 0; par < (ms.multi ? 2 : 1); ++par) {
        StepMaps &sm = maps.s[par];
        const __nv_bfloat16 *bhi = ms.multi ? ms.zhi[par ^ 1] : B.hi;
        const __nv_bfloat16 *blo = ms.multi ? ms.zlo[par ^ 1] : B.lo;
        if (!blo) blo = bhi;
        bool ok = opmap(&sm.b_hi, bhi, B.ld, B.rows, BN) && opmap(&sm.b_lo, blo, B.ld, B.rows, BN);
        if (e.symmetric_upper) {
            const float *D = ms.multi ? ms.z[par] : e.D;
            const float *C2 = ms.multi ? ms.z[par ^ 1] : e.C2;
            __nv_bfloat16 *Dhi = ms.multi ? ms.zhi[par] : e.Dhi;
            __nv_bfloat16 *Dlo = ms.multi ? ms.zlo[par] : e.Dlo;
            ok = ok && make_block_map(&sm.d, D, f32, 4, e.ldd, M, N);
            if (e.C || ms.multi) ok = ok && make_block_map(&sm.c, D, f32, 4, e.ldd, M, N);
            if (C2) ok = ok && make_block_map(&sm.c2, C2, f32, 4, ms.multi ? e.ldd : e.ldc2, M, N);
            if (Dhi) ok = ok && make_block_map(&sm.dhi, Dhi, b16, 2, e.ldb, M, N);
            if (Dlo) ok = ok && make_block_map(&sm.dlo, Dlo, b16, 2, e.ldb, M, N);
        }
        if (!ok) return cudaErrorInvalidValue;
    }
    const int tiles = count_tiles((M + BM - 1) / BM, (N + BN - 1) / BN, e.symmetric_upper, BN);
    // as many waves of tiles as num_sms CTAs need, over the fewest CTAs that
    // keep that count (every CTA then takes the same number of tiles; the
    // SMs left over stay free for other work, e.g. other members' launches)
    const int waves = tiles > num_sms ? (tiles + num_sms - 1) / num_sms : 1;
    const int grid = tiles > 0 ? (tiles + waves - 1) / waves : 1;
    if (!ms.multi) {
        gemm_tc_kernel<BN><<<grid, kThreads, S::kBytes, st>>>(maps, M, N, K, nsplit, g, e, ms, err);
        return cudaGetLastError();
    }
    cudaError_t r = cudaMemsetAsync(ms.bar, 0, sizeof(unsigned int), st);
    if (r != cudaSuccess) return r;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = S::kBytes;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, gemm_tc_kernel<BN>, maps, M, N, K, nsplit, g, e, ms, err);
}

template <int BN>
cudaError_t launch(int M, int N, int K, const TcOperand &A, const TcOperand &B, int nsplit, const Epilogue &e,
                   cudaStream_t st, int num_sms) {
    MultiStep ms;
    return launch<BN>(M, N, K, A, B, nsplit, e, ms, st, num_sms);
}

}  // namespace

// Tile width by a small cost model: waves of CTAs times the tile's cost,
// which grows with BN plus a fixed per-tile overhead of about 64 columns.
// Split products (nsplit = 3) fetch each hi/lo slice once below BN = 256
// (two-slot stages) but A's and B's hi parts twice at BN = 256: in the
// recurrence, whose steps wait on each other, that width costs half as much
// again.
int choose_bn(int M, int N, int sym, int num_sms, int nsplit) {
    const int cands[4] = {256, 128, 64, 32};
    int best = 256;
    long best_cost = -1;
    const int tm = (M + BM - 1) / BM;
    for (int bn : cands) {
        if (bn < 256 && N > 4096 * 2) continue;
        const int tiles = count_tiles(tm, (N + bn - 1) / bn, sym, bn);
        const long waves = (tiles + num_sms - 1) / num_sms;
        const long cost = waves * (bn + 64) * ((nsplit == 3 && bn == 256) ? 3 : 2) / 2;
        if (best_cost < 0 || cost < best_cost) {
            best_cost = cost;
            best = bn;
        }
    }
    return best;
}

template <class F>
cudaError_t dispatch_bn(int bn, F f) {
    switch (bn) {
        case 256: return f(std::integral_constant<int, 256>());
        case 128: return f(std::integral_constant<int, 128>());
        case 64: return f(std::integral_constant<int, 64>());
        default: return f(std::integral_constant<int, 32>());
    }
}

cudaError_t gemm_tc_recurrence(int p, const TcOperand &A, int nsplit, const Epilogue &e, int k_first, int k_end,
                               float *const z[2], __nv_bfloat16 *const zhi[2], __nv_bfloat16 *const zlo[2],
                               unsigned int *bar, cudaStream_t st, int num_sms, int clenshaw, int L, int *closed,
                               int kpad, const WaitPolicy &wp, const int *L_dev, uint8_t *mask_buf) {
    if (closed) *closed = 0;
    if (p <= 0 || k_end <= k_first) return cudaSuccess;
    if (!load_encode()) return cudaErrorNotSupported;
    if ((A.ld % 8) || ((uintptr_t)A.hi % 16) || !e.symmetric_upper || !e.H || !bar) return cudaErrorInvalidValue;
    if (nsplit == 3 && (!A.lo || !zlo[0] || !zlo[1])) return cudaErrorInvalidValue;
    if ((e.ldd % 4) || (e.ldh % 4) || (e.ldb % 8)) return cudaErrorInvalidValue;
    for (int i = 0; i < 2; ++i)
        if (((uintptr_t)z[i] % 16) || ((uintptr_t)zhi[i] % 16) || (zlo[i] && ((uintptr_t)zlo[i] % 16)))
            return cudaErrorInvalidValue;
    MultiStep ms;
    ms.multi = 1;
    ms.wait_cycles = wait_limit(wp);
    ms.stall = wp.stall;
    ms.L_dev = L_dev;
    if (L_dev && clenshaw) return cudaErrorInvalidValue;   // Clenshaw's sum runs from the last term down
    ms.amask = mask_buf;
    ms.k_first = k_first;
    ms.k_end = k_end;
    for (int i = 0; i < 2; ++i) {
        ms.z[i] = z[i];
        ms.zhi[i] = zhi[i];
        ms.zlo[i] = zlo[i];
    }
    ms.bar = bar;
    ms.clenshaw = clenshaw;
    ms.L = L;
    // tensor-memory resident state when every CTA owns at most one tile and
    // the state fits beside the two accumulators; the closing step of
    // Clenshaw's sum is then applied in the last step
    const int bn = choose_bn(p, p, 1, num_sms, nsplit);
    const int tiles = count_tiles((p + BM - 1) / BM, (p + bn - 1) / bn, 1, bn);
    ms.resident = (bn <= 64 && tiles <= num_sms && k_end == L) ? 1 : 0;
    TcOperand B;
    B.ld = A.ld;
    B.rows = p;
    B.hi = zhi[0];   // per-step operands come from the ring
    // operands padded with zero columns are contracted over the padded
    // length (a multiple of 128: grouped loads, no K tail)
    const int K = kpad > p ? kpad : p;
    if (K > A.ld) return cudaErrorInvalidValue;
    if (mask_buf) {
        // the K slices per stage of this launch: 2 when the grouped 3-D
        // loads apply (K a multiple of 128 below BN = 256, one product), else 1
        const int gs = (bn < 256 && K % 128 == 0 && nsplit != 3) ? 2 : 1;
        const int width = 64 * gs;
        ms.mask_groups = (K + width - 1) / width;
        amask_kernel<<<dim3(ms.mask_groups, (p + 127) / 128), 256, 0, st>>>(A.hi, A.lo, A.ld, p, K, width, mask_buf,
                                                                          ms.mask_groups);
        cudaError_t rm = cudaGetLastError();
        if (rm != cudaSuccess) return rm;
    }
    cudaError_t r2 = dispatch_bn(bn, [&](auto b) {
        return launch<decltype(b)::value>(p, p, K, A, B, nsplit, e, ms, st, num_sms);
    });
    if (r2 == cudaSuccess && closed) *closed = (ms.resident && clenshaw) ? 1 : 0;
    return r2;
}

cudaError_t gemm_tc(int M, int N, int K, const TcOperand &A, const TcOperand &B, int nsplit, const Epilogue &e,
                    cudaStream_t st, int num_sms) {
    if (M <= 0 || N <= 0 || K <= 0) return cudaSuccess;
    if (!load_encode()) return cudaErrorNotSupported;
    if ((A.ld % 8) || (B.ld % 8) || ((uintptr_t)A.hi % 16) || ((uintptr_t)B.hi % 16)) return cudaErrorInvalidValue;
    if (nsplit == 3 && (!A.lo || !B.lo)) return cudaErrorInvalidValue;
    if (e.symmetric_upper) {
        // the epilogue block maps need 16-byte aligned rows and bases
        if (M != N) return cudaErrorInvalidValue;
        if ((e.ldd % 4) || (e.C && e.ldc % 4) || (e.C2 && e.ldc2 % 4) || (e.H && e.ldh % 4) ||
            (e.Dhi && e.ldb % 8) || ((uintptr_t)e.D % 16) || ((uintptr_t)e.C % 16) || ((uintptr_t)e.C2 % 16) ||
            ((uintptr_t)e.H % 16) || ((uintptr_t)e.Dhi % 16) || ((uintptr_t)e.Dlo % 16))
            return cudaErrorInvalidValue;
        // C, when given, is updated in place (D == C)
        if (e.C && (e.C != e.D || e.ldc != e.ldd)) return cudaErrorInvalidValue;
    } else if (e.C || e.C2 || e.H || e.Dhi || e.Dlo) {
        return cudaErrorInvalidValue;   // general outputs carry only D
    }
    // single products keep the plain model: at BN = 256 their many waves
    // amortise the second fetch (measured on the 4096 x 8192 Gram and apply)
    return dispatch_bn(choose_bn(M, N, e.symmetric_upper, num_sms, 1), [&](auto bn) {
        return launch<decltype(bn)::value>(M, N, K, A, B, nsplit, e, st, num_sms);
    });
}

}  // namespace cpa
