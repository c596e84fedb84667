// Persistent batch kernel: one launch advances every instance of a batch by one Runge-Kutta
// step (both stages of Sec. 2.3).
//
// The work of a step is a queue of items (stage, pass, size group, instance, tile), ordered
// by stage and pass first: the column tiles of every instance's first stage, then its macro
// row blocks, its flux column tiles, its update row blocks, then the same for the second stage.
// CTAs of a persistent grid take the next item from a global counter. For one instance the
// eight passes of a step form a chain (each reads what the previous one wrote), so an item
// waits until every tile of the previous pass of its own instance has reported completion in
// a per-instance counter; instances never wait for one another, so different instances are at
// different passes at the same time and the tail of one pass overlaps the start of the next.
// Since items are taken in queue order and an item only waits for items earlier in the queue,
// each awaited item is already held by a running CTA, which completes it.
//
// Every wait is bounded (a clock-cycle budget): a wait that runs out sets the batch's abort
// flag and error word, and every CTA then leaves at its next wait; lbm_batch_synchronize
// reports LBM_ERR_TIMEOUT. Data written by other CTAs during the launch is read L2-only (the
// pass bodies use ld.global.cg for it), so no stale L1 line is ever read.
#include "pass_bodies.cuh"

namespace lbm {

__device__ __forceinline__ int ld_acquire(const int *p) {
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// the tile bodies of one pass for the line lengths the batch kernel takes (128 .. 1024 points)
#define LBM_BATCH_LOG2N(X) X(7) X(8) X(9) X(10)

template <typename R>
__device__ __forceinline__ void batch_col(const ColArgs<R> &c, int tiles_x, int tile, int z) {
    const int job = tile / tiles_x, tx = tile % tiles_x;
    switch (c.ay.log2n) {
#define LBM_CASE(L2) \
    case L2: col_tile<R, L2, 1, true>(c, job, z, tx, 0u); break;
        LBM_BATCH_LOG2N(LBM_CASE)
#undef LBM_CASE
    }
}

template <typename R> __device__ __forceinline__ void batch_macro(const MacroArgs<R> &m, int blk) {
    switch (m.ax.log2n) {
#define LBM_CASE(L2) \
    case L2: macro_rows<R, L2, false, true>(m, blk); break;
        LBM_BATCH_LOG2N(LBM_CASE)
#undef LBM_CASE
    }
}

template <typename R>
__device__ __forceinline__ void batch_update(const UpdateArgs<R> &u, const UpdateConst<R> &kc, int blk) {
    switch (u.ax.log2n) {
#define LBM_CASE(L2) \
    case L2: update_rows<R, L2, sizeof(R) == 4, 1>(u, kc, blk, 0u); break;
        LBM_BATCH_LOG2N(LBM_CASE)
#undef LBM_CASE
    }
}

// TPB threads per CTA (512 or 256), at least MINB CTAs per SM (the register budget)
template <typename R, int TPB, int MINB>
__global__ void __launch_bounds__(TPB, MINB) batch_step_kernel(const __grid_constant__ BatchArgs<R> a) {
    __shared__ int s_item, s_ok;
    const int total = a.seg[kBatchPasses * a.ngroups];
    int *queue = a.ctrl, *abort_flag = a.ctrl + 1, *done = a.ctrl + 2;
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(queue, 1);
        __syncthreads();
        const int item = s_item;
        if (item >= total) return;  // uniform: the whole CTA read the same item
        int sg = 0;
        while (a.seg[sg + 1] <= item) ++sg;
        const int chain = sg / a.ngroups, gi = sg % a.ngroups;  // chain = 4 stage + pass
        const int pass = chain & 3, stage = chain >> 2;
        const BatchGroup<R> &G = a.g[gi];
        const int j = item - a.seg[sg], nt = G.ntile[pass];
        const int k = j / nt, tile = j % nt;
        int *cnt = done + (G.inst0 + k) * kBatchPasses;
        if (threadIdx.x == 0) {
            bool ok = true;
            if (chain > 0) {
                const int need = G.ntile[(pass + 3) & 3];  // every tile of the previous pass of this instance
                const long long t0 = clock64();
                while (ld_acquire(cnt + chain - 1) < need) {
                    if (ld_acquire(abort_flag) || clock64() - t0 > a.wait_cycles) {
                        ok = false;
                        break;
                    }
                    __nanosleep(100);
                }
            }
            if (!ok) {
                atomicExch(abort_flag, 1);
                atomicOr(a.err, tma::kErrTimeout);
            }
            s_ok = ok ? 1 : 0;
        }
        __syncthreads();
        if (!s_ok) return;  // uniform
        switch (pass) {
            case 0: batch_col<R>(G.col[stage], G.tiles_x[0], tile, k); break;
            case 1: batch_macro<R>(G.macro, k * G.ntile[1] + tile); break;
            case 2: batch_col<R>(G.flux[stage], G.tiles_x[1], tile, k); break;
            default: batch_update<R>(G.upd[stage], G.upd[stage].k, k * G.ntile[3] + tile); break;
        }
        __syncthreads();  // every thread's results of this item are written
        if (threadIdx.x == 0 && !(a.withhold && item == 0)) {
            __threadfence();
            atomicAdd(cnt + chain, 1);
        }
    }
}

template <typename R, int TPB, int MINB> cudaError_t launch_batch_tpb(const BatchArgs<R> &a, size_t smem, int grid,
                                                                       cudaStream_t s) {
    cudaError_t e = allow_smem(batch_step_kernel<R, TPB, MINB>);
    if (e != cudaSuccess) return e;
    batch_step_kernel<R, TPB, MINB><<<grid, TPB, smem, s>>>(a);
    return cudaGetLastError();
}

template <typename R> cudaError_t launch_batch_step(const BatchArgs<R> &a, size_t smem, int grid, int tpb,
                                                   cudaStream_t s) {
    if (tpb == 256) return launch_batch_tpb<R, 256, 3>(a, smem, grid, s);
    if (tpb == 512) return launch_batch_tpb<R, 512, 2>(a, smem, grid, s);
    return cudaErrorInvalidValue;
}

template <typename R> cudaError_t batch_step_ctas_per_sm(size_t smem, int tpb, int *n) {
    *n = 0;
    cudaError_t e;
    if (tpb == 256) {
        if ((e = allow_smem(batch_step_kernel<R, 256, 3>)) != cudaSuccess) return e;
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(n, batch_step_kernel<R, 256, 3>, 256, smem);
    }
    if (tpb == 512) {
        if ((e = allow_smem(batch_step_kernel<R, 512, 2>)) != cudaSuccess) return e;
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(n, batch_step_kernel<R, 512, 2>, 512, smem);
    }
    return cudaErrorInvalidValue;
}

template cudaError_t launch_batch_step<float>(const BatchArgs<float> &, size_t, int, int, cudaStream_t);
template cudaError_t batch_step_ctas_per_sm<float>(size_t, int, int *);

}  // namespace lbm
