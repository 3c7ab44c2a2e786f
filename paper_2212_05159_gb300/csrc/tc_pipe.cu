// Pipelined tensor-core kernel for the network's dense layers: the forward product
// Y = [X1 X2] W + b with its epilogues, and the data gradient [dX1 dX2] (+)= G W^T.  Same
// arithmetic as the kernels of tc_dense.cu (A rounded to BF16, BF16 weights, the same K/16
// tcgen05.mma steps accumulating in FP32 in tensor memory, the same epilogue operations),
// so the results are bitwise equal; this kernel only moves the data differently.
//
// One persistent CTA per SM walks 128-row tiles with four warp roles:
//   warp 0      (one thread) TMA producer: the tile's FP32 rows of each source matrix as
//               boxes of 32 columns x 128 rows (cp.async.bulk.tensor, 128-byte swizzle, rows
//               past n filled with zeros) into a ring of S stages, completion counted in
//               bytes on the stage's "full" mbarrier;
//   warps 1-4   converters: FP32 stage -> BF16 operand tile in the canonical no-swizzle
//               K-major core-matrix layout (thread = row; the swizzle makes both the stage
//               reads and the core-matrix writes conflict-free), then one arrive per warp;
//   warp 5      (one thread) issues the K/16 MMAs of a tile into one of two accumulators in
//               tensor memory and commits them to the "operand free" and "accumulator full"
//               mbarriers (warp 5 also allocates and frees the tensor memory);
//   warps 6-9   epilogue: warp w reads accumulator lanes 32 (w mod 4) .. + 31 (its rows)
//               with tcgen05.ld, 32 columns at a time, releases the accumulator after its
//               last read, applies bias / relu / residual (the residual rows read from the
//               stage when Hin is X1, else from global memory), writes each 32 x 32 block
//               into a swizzled shared-memory slot and stores it with a TMA tensor store
//               (reduce-add for an accumulating data gradient: old + new, one rounding, as
//               a load-add-store), rows past n clipped by the TMA; it releases the stage
//               after its last residual read.
// Every wait is bounded (2 s): a wait that runs out sets a flag that ends every role's
// loop, records a device error, and the roles drain their own TMA copies and MMAs (again
// with bounded waits) before warp 5 frees the tensor memory.
#include <cuda.h>
#include <cuda_bf16.h>

#include <atomic>
#include <mutex>

#include "common.cuh"
#include "tc_pipe.h"

namespace spx {
namespace {

constexpr int TP_M = 128;                        // rows per tile (the MMA's M)
constexpr int TP_THREADS = 320;                  // 10 warps
constexpr int TP_BOX_COLS = 32;                  // FP32 columns per TMA box (128 bytes)
constexpr int TP_IN_BOX = TP_M * 128;            // one input box: 128 rows x 128 B = 16 KB
constexpr int TP_OUT_BOX = 32 * 128;             // one output box: 32 rows x 128 B = 4 KB
constexpr int TP_MAX_STAGES = 4;
constexpr int TP_SMEM_LIMIT = 227 * 1024;
constexpr uint64_t TP_WAIT_NS = 2000000000ull;

enum TpKind : int { TP_FORWARD = 0, TP_BWD_DATA = 1 };

struct TpParams {
    int64_t n;
    int kind;          // TpKind
    int K1, K2;        // A-source column counts (forward: X1, X2; data gradient: N, 0)
    int kpad;          // K1 + K2 (a multiple of 32)
    int nout;          // the MMA's N: forward N; data gradient K1 + K2 of the outputs
    int ncols;         // tensor-memory columns per accumulator (power of two >= nout)
    int mode;          // forward epilogue mode 0..4
    int accumulate;    // data gradient: add into the outputs
    int out_split;     // columns of the first output (the rest go to the second)
    int stages, slots; // ring depth; output slots per epilogue warp
    int res_from_stage;
    int has_o2;        // the second output exists (data gradient: dX2 given)
    const __nv_bfloat16* W;
    const float* bias;
    const float* Hin;  // residual rows (global), used when !res_from_stage
    uint32_t off_stage, stage_bytes, off_op, off_b, off_out, off_bias;
    int* err;
};

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* tm, int x, int y, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            dst),
        "l"(reinterpret_cast<uint64_t>(tm)), "r"(x), "r"(y), "r"(bar)
        : "memory");
}

__device__ __forceinline__ void tma_store_2d(const CUtensorMap* tm, int x, int y, uint32_t src) {
    asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%1, %2}], [%3];" ::"l"(
                     reinterpret_cast<uint64_t>(tm)),
                 "r"(x), "r"(y), "r"(src)
                 : "memory");
}

__device__ __forceinline__ void tma_reduce_add_2d(const CUtensorMap* tm, int x, int y, uint32_t src) {
    asm volatile("cp.reduce.async.bulk.tensor.2d.global.shared::cta.add.bulk_group [%0, {%1, %2}], [%3];" ::"l"(
                     reinterpret_cast<uint64_t>(tm)),
                 "r"(x), "r"(y), "r"(src)
                 : "memory");
}

__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void bulk_wait_read() {
    asm volatile("cp.async.bulk.wait_group.read %0;" ::"n"(N) : "memory");
}
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

__device__ __forceinline__ uint64_t tp_smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((addr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;                       // descriptor version of the sm_100 family
    return d;                                     // base offset 0, no swizzle
}

// kind::f16 instruction descriptor: D F32, A and B BF16, both K-major, M x N.
__device__ __forceinline__ uint32_t tp_instr_desc(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// byte offset of element (row, k) in the core-matrix layout of a rows x kpad operand
__device__ __forceinline__ uint32_t tp_core_off(int row, int k, int kpad) {
    return (uint32_t)((row >> 3) * (kpad >> 3) * 128 + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2);
}

// byte offset of the 16-byte chunk `ch` (0..7) of row `row` in a 128-byte-swizzled box
__device__ __forceinline__ uint32_t swz(int row, int ch) { return (uint32_t)(row * 128 + ((ch ^ (row & 7)) << 4)); }

__device__ __forceinline__ uint32_t pack2(float a, float b) {
    __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<uint32_t*>(&h);
}

// A bounded wait shared by the roles: gives up when another role has already given up.
__device__ __forceinline__ bool tp_wait(uint32_t bar, uint32_t parity, volatile int* abort_flag) {
    if (*abort_flag) return false;
    const uint64_t t0 = global_ns();
    for (;;) {
        uint32_t ok;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(bar), "r"(parity)
            : "memory");
        if (ok) return true;
        if (*abort_flag) return false;
        if (global_ns() - t0 > TP_WAIT_NS) {
            *abort_flag = 1;
            return false;
        }
    }
}

// 32 consecutive accumulator columns of this thread's lane (row), as floats
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
    uint32_t r[32];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

__global__ void __launch_bounds__(TP_THREADS, 1)
    tc_pipe_kernel(const __grid_constant__ CUtensorMap tmA1, const __grid_constant__ CUtensorMap tmA2,
                   const __grid_constant__ CUtensorMap tmO1, const __grid_constant__ CUtensorMap tmO2, TpParams p) {
    extern __shared__ unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t bar_full[TP_MAX_STAGES], bar_empty[TP_MAX_STAGES];
    __shared__ __align__(8) uint64_t bar_op_full, bar_op_empty, bar_acc_full[2], bar_acc_empty[2];
    __shared__ uint32_t tmem_slot;
    __shared__ int abort_flag;
    // 1 KB-aligned base (the 128-byte swizzle repeats every 1024 bytes)
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    unsigned char* sm = smem_raw + (base - raw);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t ntiles = (p.n + TP_M - 1) / TP_M;
    const int kpad = p.kpad;
    const int nbox1 = p.K1 / TP_BOX_COLS, nbox = kpad / TP_BOX_COLS;

    // ---- once per CTA: B operand (K-major over the reduction), bias, barriers, tensor memory
    unsigned char* sB = sm + p.off_b;
    for (int t = threadIdx.x; t < p.nout * kpad; t += TP_THREADS) {
        // forward: B row j = column j of W (K x N); data gradient: B row j = row j of W (outputs x N)
        const int row = p.kind == TP_FORWARD ? t % p.nout : t / kpad;
        const int k = p.kind == TP_FORWARD ? t / p.nout : t % kpad;
        const __nv_bfloat16 w = p.kind == TP_FORWARD ? p.W[(size_t)k * p.nout + row] : p.W[(size_t)row * kpad + k];
        *reinterpret_cast<__nv_bfloat16*>(sB + tp_core_off(row, k, kpad)) = w;
    }
    float* sbias = reinterpret_cast<float*>(sm + p.off_bias);
    for (int t = threadIdx.x; t < p.nout; t += TP_THREADS) sbias[t] = p.bias ? p.bias[t] : 0.f;
    if (threadIdx.x == 0) {
        for (int s = 0; s < p.stages; ++s) {
            mbar_init(smem_u32(&bar_full[s]), 1);
            mbar_init(smem_u32(&bar_empty[s]), 4);
        }
        mbar_init(smem_u32(&bar_op_full), 4);
        mbar_init(smem_u32(&bar_op_empty), 1);
        for (int a = 0; a < 2; ++a) {
            mbar_init(smem_u32(&bar_acc_full[a]), 1);
            mbar_init(smem_u32(&bar_acc_empty[a]), 4);
        }
        abort_flag = 0;
        fence_mbar_init();
    }
    if (warp == 5) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                     "r"(2 * p.ncols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_proxy_async();                          // B written by the generic proxy, read by the MMAs
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_slot;
    volatile int* abort_v = &abort_flag;

    if (warp == 0) {
        // ================= TMA producer
        if (lane == 0) {
            asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmA1)) : "memory");
            if (p.K2 > 0) asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmA2)) : "memory");
            int64_t issued = 0;
            for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++issued) {
                const int s = (int)(issued % p.stages);
                const uint32_t ph = (uint32_t)((issued / p.stages) & 1);
                if (!tp_wait(smem_u32(&bar_empty[s]), ph ^ 1u, abort_v)) break;
                const uint32_t full = smem_u32(&bar_full[s]);
                const uint32_t dst = base + p.off_stage + (uint32_t)s * p.stage_bytes;
                mbar_arrive_expect_tx(full, (uint32_t)(nbox * TP_IN_BOX));
                const int y = (int)(tile * TP_M);
                for (int b = 0; b < nbox1; ++b) tma_load_2d(dst + b * TP_IN_BOX, &tmA1, b * TP_BOX_COLS, y, full);
                for (int b = nbox1; b < nbox; ++b)
                    tma_load_2d(dst + b * TP_IN_BOX, &tmA2, (b - nbox1) * TP_BOX_COLS, y, full);
            }
            // drain: the copies of the last (up to S) issued tiles have landed before the CTA
            // may end (on the normal path these waits return at once)
            for (int64_t q = issued - p.stages < 0 ? 0 : issued - p.stages; q < issued; ++q) {
                const int s = (int)(q % p.stages);
                mbar_wait(smem_u32(&bar_full[s]), (uint32_t)((q / p.stages) & 1), TP_WAIT_NS);
            }
        }
    } else if (warp <= 4) {
        // ================= converters: thread = tile row
        const int row = threadIdx.x - 32;
        unsigned char* op = sm + p.off_op;
        int64_t it = 0;
        for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++it) {
            const int s = (int)(it % p.stages);
            const uint32_t ph = (uint32_t)((it / p.stages) & 1);
            bool ok = tp_wait(smem_u32(&bar_full[s]), ph, abort_v);
            ok = ok && tp_wait(smem_u32(&bar_op_empty), (uint32_t)(it & 1) ^ 1u, abort_v);
            if (!__all_sync(FULL, ok)) break;
            const unsigned char* st = sm + p.off_stage + (size_t)s * p.stage_bytes + row * 128;
#pragma unroll 4
            for (int k8 = 0; k8 < kpad / 8; ++k8) {
                const unsigned char* bp = st + (k8 >> 2) * TP_IN_BOX;
                const int ch = (k8 & 3) * 2;
                const float4 a = *reinterpret_cast<const float4*>(bp + ((ch ^ (row & 7)) << 4));
                const float4 b = *reinterpret_cast<const float4*>(bp + (((ch + 1) ^ (row & 7)) << 4));
                *reinterpret_cast<uint4*>(op + tp_core_off(row, k8 * 8, kpad)) =
                    make_uint4(pack2(a.x, a.y), pack2(a.z, a.w), pack2(b.x, b.y), pack2(b.z, b.w));
            }
            fence_proxy_async();                  // operand writes -> visible to the tensor cores
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(&bar_op_full));
        }
    } else if (warp == 5) {
        // ================= MMA issuer
        if (lane == 0) {
            const uint32_t idesc = tp_instr_desc(TP_M, p.nout);
            const uint32_t a0 = base + p.off_op, b0 = base + p.off_b;
            const uint32_t sbo = (uint32_t)(kpad >> 3) * 128u;
            int64_t it = 0;
            for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++it) {
                const int a = (int)(it & 1);
                const uint32_t use = (uint32_t)((it >> 1) & 1);
                if (!tp_wait(smem_u32(&bar_op_full), (uint32_t)(it & 1), abort_v)) break;
                if (!tp_wait(smem_u32(&bar_acc_empty[a]), use ^ 1u, abort_v)) break;
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t d = tmem + (uint32_t)(a * p.ncols);
                for (int s = 0; s < kpad / 16; ++s) {
                    const uint64_t ad = tp_smem_desc(a0 + s * 256u, 128u, sbo);
                    const uint64_t bd = tp_smem_desc(b0 + s * 256u, 128u, sbo);
                    const uint32_t acc = s > 0 ? 1u : 0u;
                    asm volatile(
                        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
                        "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
                        : "memory");
                }
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                 smem_u32(&bar_op_empty))
                             : "memory");
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                 smem_u32(&bar_acc_full[a]))
                             : "memory");
            }
            // drain: the last tile's MMAs have completed before the tensor memory is freed
            if (it > 0) mbar_wait(smem_u32(&bar_op_empty), (uint32_t)((it - 1) & 1), TP_WAIT_NS);
        }
    } else {
        // ================= epilogue: warp w owns tile rows 32 (w mod 4) .. + 31, thread = row
        const int q = warp & 3, ew = warp - 6;
        const int r = 32 * q + lane;
        const uint32_t slot_base = base + p.off_out + (uint32_t)(ew * p.slots) * TP_OUT_BOX;
        unsigned char* slot_ptr = sm + p.off_out + (size_t)(ew * p.slots) * TP_OUT_BOX;
        const bool fwd = p.kind == TP_FORWARD;
        int64_t nb = 0;                                      // boxes stored by this warp
        int64_t it = 0;
        for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++it) {
            const int s = (int)(it % p.stages);
            const int a = (int)(it & 1);
            const uint32_t use = (uint32_t)((it >> 1) & 1);
            const bool ok = tp_wait(smem_u32(&bar_acc_full[a]), use, abort_v);
            if (!__all_sync(FULL, ok)) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const int64_t row0 = tile * TP_M;
            const int64_t grow = row0 + 32 * q;              // first row of this warp's boxes
            const bool live = grow < p.n;                    // warp-uniform
            const unsigned char* st = sm + p.off_stage + (size_t)s * p.stage_bytes;
            // one 32 x 32 block of output (this thread's row, 32 columns) to a tensor map
            auto emit = [&](const CUtensorMap* tm, int col, const float (&o)[32], bool reduce) {
                if (!live) return;
                const int slot = (int)(nb % p.slots);
                if (nb >= p.slots) {                         // the slot's previous store has read it
                    if (lane == 0) {
                        if (p.slots == 4) bulk_wait_read<3>();
                        else bulk_wait_read<1>();
                    }
                    __syncwarp();
                }
                unsigned char* sp = slot_ptr + slot * TP_OUT_BOX;
#pragma unroll
                for (int ch = 0; ch < 8; ++ch)
                    *reinterpret_cast<float4*>(sp + swz(lane, ch)) =
                        make_float4(o[4 * ch], o[4 * ch + 1], o[4 * ch + 2], o[4 * ch + 3]);
                fence_proxy_async();                         // slot writes -> visible to the TMA
                __syncwarp();
                if (lane == 0) {
                    const uint32_t src = slot_base + (uint32_t)slot * TP_OUT_BOX;
                    if (reduce) tma_reduce_add_2d(tm, col, (int)grow, src);
                    else tma_store_2d(tm, col, (int)grow, src);
                    bulk_commit();
                }
                ++nb;
            };
            for (int j0 = 0; j0 < p.nout; j0 += 32) {
                float v[32];
                tmem_ld32(tmem + (uint32_t)(a * p.ncols) + ((uint32_t)(32 * q) << 16) + (uint32_t)j0, v);
                if (j0 + 32 >= p.nout) {                     // the accumulator is free for tile it + 2
                    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                    __syncwarp();
                    if (lane == 0) mbar_arrive(smem_u32(&bar_acc_empty[a]));
                }
                if (!fwd) {
                    if (j0 < p.out_split) emit(&tmO1, j0, v, p.accumulate != 0);
                    else if (p.has_o2) emit(&tmO2, j0 - p.out_split, v, p.accumulate != 0);
                    continue;
                }
#pragma unroll
                for (int c = 0; c < 32; ++c) v[c] = v[c] + sbias[j0 + c];
                if (p.mode == 0) {
                    emit(&tmO1, j0, v, false);
                } else if (p.mode == 1) {
#pragma unroll
                    for (int c = 0; c < 32; ++c) v[c] = fmaxf(v[c], 0.f);
                    emit(&tmO1, j0, v, false);
                } else if (p.mode == 4) {
                    if (j0 < p.out_split) emit(&tmO1, j0, v, false);
                    else emit(&tmO2, j0 - p.out_split, v, false);
                } else {
                    float h[32];
                    if (p.res_from_stage) {
                        const unsigned char* hb = st + (j0 / TP_BOX_COLS) * TP_IN_BOX;
#pragma unroll
                        for (int ch = 0; ch < 8; ++ch) {
                            const float4 t = *reinterpret_cast<const float4*>(hb + swz(r, ch));
                            h[4 * ch] = t.x;
                            h[4 * ch + 1] = t.y;
                            h[4 * ch + 2] = t.z;
                            h[4 * ch + 3] = t.w;
                        }
                    } else {
                        const int64_t grow_t = row0 + r;
#pragma unroll
                        for (int ch = 0; ch < 8; ++ch) {
                            float4 t = make_float4(0.f, 0.f, 0.f, 0.f);
                            if (grow_t < p.n)
                                t = __ldcs(reinterpret_cast<const float4*>(p.Hin + grow_t * p.nout + j0 + 4 * ch));
                            h[4 * ch] = t.x;
                            h[4 * ch + 1] = t.y;
                            h[4 * ch + 2] = t.z;
                            h[4 * ch + 3] = t.w;
                        }
                    }
                    if (p.mode == 2) emit(&tmO2, j0, v, false);     // U = the pre-activation
#pragma unroll
                    for (int c = 0; c < 32; ++c) h[c] = h[c] + fmaxf(v[c], 0.f);
                    emit(&tmO1, j0, h, false);
                }
            }
            __syncwarp();                                    // residual reads of stage s done
            if (lane == 0) mbar_arrive(smem_u32(&bar_empty[s]));
        }
        if (lane == 0) bulk_wait_all();                      // stores complete before the CTA ends
        __syncwarp();
    }

    // ---- teardown: every role has left its loop and drained its own asynchronous work
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (threadIdx.x == 0 && *abort_v && p.err) atomicOr(p.err, 2);
    if (warp == 5) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * p.ncols) : "memory");
    }
}

// ------------------------------------------------------------------ host side
std::atomic<int> g_pipe_enabled{1};

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

spx_status encode_fn(EncodeTiledFn* out) {
    static std::mutex mu;
    static EncodeTiledFn fn = nullptr;
    std::lock_guard<std::mutex> lock(mu);
    if (!fn) {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        SPX_CUDA(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q),
                 "tensor map: driver entry point cuTensorMapEncodeTiled");
        if (q != cudaDriverEntryPointSuccess || !f)
            return set_error(SPX_NOT_SUPPORTED, "tensor map: the driver lacks cuTensorMapEncodeTiled");
        fn = reinterpret_cast<EncodeTiledFn>(f);
    }
    *out = fn;
    return SPX_OK;
}

// A row-major FP32 matrix (rows x cols, row stride cols) as 2-D tiles of box_cols x
// box_rows with the 128-byte swizzle; rows beyond the matrix read as zeros and are not written.
spx_status encode_f32(CUtensorMap* tm, const float* ptr, int64_t rows, int cols, int box_rows) {
    EncodeTiledFn fn = nullptr;
    SPX_TRY(encode_fn(&fn));
    const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)cols * 4};
    const cuuint32_t box[2] = {(cuuint32_t)TP_BOX_COLS, (cuuint32_t)box_rows};
    const cuuint32_t estr[2] = {1, 1};
    const CUresult r = fn(tm, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(ptr), dims, strides, box, estr,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS)
        return set_error(SPX_CUDA_ERROR, "cuTensorMapEncodeTiled failed (%d) for a %lld x %d matrix", (int)r,
                         (long long)rows, cols);
    return SPX_OK;
}

inline uint32_t al1k(uint32_t x) { return (x + 1023u) & ~1023u; }

// Shared-memory layout for a ring of `stages` and `slots` output slots per epilogue warp;
// false if it does not fit.
bool tp_layout(TpParams& p, int stages, int slots) {
    const uint32_t nbox = (uint32_t)(p.kpad / TP_BOX_COLS);
    p.stages = stages;
    p.slots = slots;
    p.off_stage = 0;
    p.stage_bytes = nbox * TP_IN_BOX;
    p.off_op = p.off_stage + (uint32_t)stages * p.stage_bytes;
    p.off_b = al1k(p.off_op + (uint32_t)TP_M * p.kpad * 2);
    p.off_out = al1k(p.off_b + (uint32_t)p.nout * p.kpad * 2);
    p.off_bias = p.off_out + 4u * (uint32_t)slots * TP_OUT_BOX;
    const uint32_t total = p.off_bias + 512u + 1024u;           // bias; 1 KB alignment slack
    return total <= (uint32_t)(TP_SMEM_LIMIT - 1024);
}

uint32_t tp_smem_bytes(const TpParams& p) { return p.off_bias + 512u + 1024u; }

spx_status tp_launch(TpParams& p, const CUtensorMap& a1, const CUtensorMap& a2, const CUtensorMap& o1,
                     const CUtensorMap& o2, cudaStream_t st) {
    bool fits = false;
    for (int slots : {4, 2}) {
        for (int stages = TP_MAX_STAGES; stages >= 2 && !fits; --stages) fits = tp_layout(p, stages, slots);
        if (fits) break;
    }
    if (!fits) return set_error(SPX_NOT_SUPPORTED, "tensor-core pipeline: shared memory");
    static std::atomic<unsigned long long> attr_done{0};
    SPX_TRY(ensure_smem_attr(tc_pipe_kernel, TP_SMEM_LIMIT - 1024, attr_done, "tensor-core pipeline attribute"));
    const int64_t tiles = (p.n + TP_M - 1) / TP_M;
    const int64_t grid = tiles < num_sms() ? tiles : num_sms();
    p.err = device_error_word();
    tc_pipe_kernel<<<(unsigned)grid, TP_THREADS, tp_smem_bytes(p), st>>>(a1, a2, o1, o2, p);
    SPX_CHECK_LAUNCH("tensor-core pipeline");
    return SPX_OK;
}

int pow2_cols(int n) { return n <= 32 ? 32 : (n <= 64 ? 64 : 128); }

}  // namespace

bool tc_pipe_enabled() { return g_pipe_enabled.load(std::memory_order_relaxed) != 0; }

spx_status tc_pipe_forward(int64_t n, const float* X1, int K1, const float* X2, int K2, const __nv_bfloat16* W,
                           const float* bias, int N, int mode, const float* Hin, float* Y, float* U, cudaStream_t st,
                           bool* launched) {
    *launched = false;
    if (!tc_pipe_enabled() || n < 1 || n >= (int64_t)INT32_MAX - TP_M) return SPX_OK;
    if (K1 < 32 || K1 % 32 != 0 || K2 % 32 != 0 || K1 + K2 > 128 || N < 32 || N > 128 || N % 32 != 0) return SPX_OK;
    if (mode == 4 && (N / 2) % 32 != 0) return SPX_OK;
    TpParams p{};
    p.n = n;
    p.kind = TP_FORWARD;
    p.K1 = K1;
    p.K2 = K2;
    p.kpad = K1 + K2;
    p.nout = N;
    p.ncols = pow2_cols(N);
    p.mode = mode;
    p.W = W;
    p.bias = bias;
    p.Hin = Hin;
    p.res_from_stage = (mode == 2 || mode == 3) && Hin == X1 && K1 == N;
    p.out_split = mode == 4 ? N / 2 : N;
    p.has_o2 = mode == 2 || mode == 4;
    CUtensorMap a1, a2, o1, o2;
    SPX_TRY(encode_f32(&a1, X1, n, K1, TP_M));
    if (K2 > 0) SPX_TRY(encode_f32(&a2, X2, n, K2, TP_M));
    else a2 = a1;
    const int ny = mode == 4 ? N / 2 : N;
    SPX_TRY(encode_f32(&o1, Y, n, ny, 32));
    if (p.has_o2) SPX_TRY(encode_f32(&o2, U, n, ny, 32));
    else o2 = o1;
    SPX_TRY(tp_launch(p, a1, a2, o1, o2, st));
    *launched = true;
    return SPX_OK;
}

spx_status tc_pipe_bwd_data(int64_t n, const float* G, int N, const __nv_bfloat16* W, int K1, int K2, float* dX1,
                            float* dX2, int accumulate, cudaStream_t st, bool* launched) {
    *launched = false;
    if (!tc_pipe_enabled() || n < 1 || n >= (int64_t)INT32_MAX - TP_M) return SPX_OK;
    if (N < 32 || N > 128 || N % 32 != 0 || K1 < 32 || K1 % 32 != 0 || K2 % 32 != 0 || K1 + K2 > 128) return SPX_OK;
    TpParams p{};
    p.n = n;
    p.kind = TP_BWD_DATA;
    p.K1 = N;                           // the A source is G (n x N)
    p.K2 = 0;
    p.kpad = N;
    p.nout = K1 + K2;
    p.ncols = pow2_cols(K1 + K2);
    p.accumulate = accumulate;
    p.W = W;
    p.out_split = K1;
    p.has_o2 = K2 > 0 && dX2 != nullptr;
    CUtensorMap a1, o1, o2;
    SPX_TRY(encode_f32(&a1, G, n, N, TP_M));
    SPX_TRY(encode_f32(&o1, dX1, n, K1, 32));
    if (p.has_o2) SPX_TRY(encode_f32(&o2, dX2, n, K2, 32));
    else o2 = o1;
    SPX_TRY(tp_launch(p, a1, a1, o1, o2, st));
    *launched = true;
    return SPX_OK;
}

}  // namespace spx

extern "C" spx_status spx_tc_set_pipeline(int32_t enabled) {
    spx::g_pipe_enabled.store(enabled ? 1 : 0, std::memory_order_relaxed);
    return SPX_OK;
}
