// wcc_batch.cuh -- many independent 1D problems advanced by one persistent
// launch per half-step (FP32-mixed).
//
// The instances of a batch share the conservation law and the options; each
// has its own N, P, domain, boundary and dt (from its own CFL bound).  Cells
// are flattened, not instances: every instance is cut into tiles of kTile new
// cells (kTileMixed for the half-step, kTile for the auxiliary kernels), the
// tiles of all instances form one list (prefix table tile_start), and a
// persistent grid walks the list.  A launch covers two
// groups of instances, P = PA and P = PB (a batch holds at most two degrees);
// each group keeps its stages in its own plane buffers with instance
// offsets.  The tile code is the single-grid kernel's (mixed_tile), so an
// instance of a batch evolves exactly like the same problem run alone.
#pragma once

#include "wcc_convert.cuh"
#include "wcc_mixed2.cuh"

namespace wcc {

struct BatchInstance {
    long long offset;     // first cell of the instance in its group's planes
    long long aos_offset[2];  // first double of the instance in the host-layout array of a stage of parity 0 / 1
    long long cells[2];   // cells of an integer (0) / half (1) stage
    double dx;
    int bc;
    int group;            // 0: P = PA, 1: P = PB
};

struct BatchArgs {
    StepArgs phys;                 // physics and options (per-launch fields unused)
    const BatchInstance* inst;
    DevState* st;                  // one per instance
    double* hist;                  // hist[i * hist_cap + step]
    long long hist_cap;
    const float* in[2];            // current stage planes of group 0 / 1
    float* out[2];                 // next stage planes
    long long pitch[2];
    const long long* tile_start;   // [ninst + 1] exclusive prefix of tiles per instance
    const int* tile_inst;          // [total_tiles] instance of every tile
    long long total_tiles;
    int ninst;
    int parity;
    // two half-steps per launch: the second half-step's largest CFL number
    // per group, the states before the launch, the batch's refusal flag
    double nu_max[2];
    DevState* tb_backup;
    unsigned* tb_refused;
};


template <int SYS, int PA, int PB>
__global__ void __launch_bounds__(kThreadsMixed, (mixed_min_ctas<PA>() < mixed_min_ctas<PB>() ? mixed_min_ctas<PA>()
                                                                                            : mixed_min_ctas<PB>()))
    batch_mixed(const BatchArgs b) {
    constexpr int SA = mixed2_smem_float2<SYS, PA>();
    constexpr int SB = mixed2_smem_float2<SYS, PB>();
    __shared__ float2 rec[SA > SB ? SA : SB];
    for (long long tile = blockIdx.x; tile < b.total_tiles; tile += gridDim.x) {
        const int i = __ldg(b.tile_inst + tile);
        const BatchInstance I = b.inst[i];
        DevState* st = b.st + i;
        const long long first = __ldg(b.tile_start + i);
        const long long ntiles = __ldg(b.tile_start + i + 1) - first;
        const StepSize z = cfl_step_size(st, b.phys.cfl_bits, b.phys.cfl, I.dx, b.parity);
        const int g = I.group;
        const TileIO io{b.in[g] + I.offset, b.out[g] + I.offset, b.pitch[g], I.cells[b.parity],
                        I.cells[b.parity ^ 1], (tile - first) * kTileMixed, b.parity, I.bc};
        float speed = 0.f;
        unsigned err = 0u;
        StepArgs ph = b.phys;  // per-instance boundary and mesh width
        ph.bc = I.bc;
        ph.dx = I.dx;
        // both degrees share one register budget: both park (see mixed_tile2)
        if (g == 0)
            mixed_tile2<SYS, PA, true, true>(io, ff_make(z.lam_hi, z.lam_lo), ph, rec, speed, err);
        else
            mixed_tile2<SYS, PB, true, true>(io, ff_make(z.lam_hi, z.lam_lo), ph, rec, speed, err);
        reduce_and_finish<float, kThreadsMixed>(speed, err, z.dt, st, ntiles, b.hist + (long long)i * b.hist_cap, b.hist_cap,
                                 b.parity, 1, b.phys.cfl, I.dx);
    }
}

// Two half-steps per launch for every instance (mixed_pair_tile): each
// instance is cut into tiles of kTileTB final cells (tile list in
// tile_start / tile_inst), a persistent grid walks the list, and each
// instance's last tile does the instance's pair bookkeeping (finalize_pair),
// first keeping the instance's state in tb_backup.  If any instance refuses
// its pair, the batch's flag is set and the caller restores every instance
// from tb_backup (the launch did not overwrite the input stages) and takes
// that pair as two single half-steps; launches that find the flag set do
// nothing.
template <int SYS, int PA, int PB>
__global__ void __launch_bounds__(kThreadsMixed, (mixed_min_ctas<PA>() < mixed_min_ctas<PB>() ? mixed_min_ctas<PA>()
                                                                                            : mixed_min_ctas<PB>()))
    batch_mixed_tb2(const BatchArgs b) {
    constexpr int SA = mixed2_smem_float2<SYS, PA>();
    constexpr int SB = mixed2_smem_float2<SYS, PB>();
    __shared__ float2 rec[SA > SB ? SA : SB];
    if (*(volatile unsigned*)b.tb_refused) return;
    for (long long tile = blockIdx.x; tile < b.total_tiles; tile += gridDim.x) {
        const int i = __ldg(b.tile_inst + tile);
        const BatchInstance I = b.inst[i];
        DevState* st = b.st + i;
        const long long first = __ldg(b.tile_start + i);
        const long long ntiles = __ldg(b.tile_start + i + 1) - first;
        const StepSize z = cfl_step_size(st, b.phys.cfl_bits, b.phys.cfl, I.dx, b.parity);
        const int g = I.group;
        const PairIO io{b.in[g] + I.offset, b.out[g] + I.offset, b.pitch[g], I.cells[b.parity],
                        I.cells[b.parity ^ 1], I.cells[b.parity], (tile - first) * kTileTB, b.parity, I.bc};
        StepArgs ph = b.phys;  // per-instance boundary and mesh width
        ph.bc = I.bc;
        ph.dx = I.dx;
        const ff2 lam2{f2(z.lam_hi), f2(z.lam_lo)};
        float mid = 0.f, fin = 0.f;
        unsigned err = 0u;
        // both degrees share one register budget: both park (see mixed_parent_records)
        if (g == 0)
            mixed_pair_tile<SYS, PA, true, true>(io, lam2, ph, rec, mid, fin, err);
        else
            mixed_pair_tile<SYS, PB, true, true>(io, lam2, ph, rec, mid, fin, err);
        const PairBook bk{st, b.hist + (long long)i * b.hist_cap, b.hist_cap, ntiles, I.dx, b.phys.cfl, b.nu_max[g],
                          1, b.parity, b.tb_backup + i, b.tb_refused};
        finish_pair(mid, fin, err, z.dt, bk);
    }
}

// Largest characteristic speed of every instance's current stage (after
// loading data): one thread per cell of the tiles in tile_start (tiles of
// the current stage), into st[i].amax_bits[parity].
template <int SYS, int PA, int PB>
__global__ void __launch_bounds__(kThreads) batch_stage_speed(const BatchArgs b) {
    for (long long tile = blockIdx.x; tile < b.total_tiles; tile += gridDim.x) {
        const int i = __ldg(b.tile_inst + tile);
        const BatchInstance I = b.inst[i];
        const long long c = (tile - b.tile_start[i]) * kTile + threadIdx.x;
        float s = 0.f;
        unsigned err = 0u;
        if (threadIdx.x < kTile && c < I.cells[b.parity]) {
            const int P = I.group == 0 ? PA : PB;
            const int NP = P + 2;
            const float* pl = b.in[I.group] + I.offset;
            const long long pitch = b.pitch[I.group];
            float u0[nvars(SYS)];
#pragma unroll
            for (int v = 0; v < nvars(SYS); ++v) {
                float corr = 0.f;
                for (int k = 2; k <= P; k += 2)
                    corr += pl[(long long)(v * NP + k + 1) * pitch + c] / (float)((k + 1) * (1 << k));
                u0[v] = (pl[(long long)(v * NP) * pitch + c] + pl[(long long)(v * NP + 1) * pitch + c]) - corr;
            }
            StepArgs ph = b.phys;
            s = wave_speed<SYS, float>(u0, ph, err);
            if (s != s) {
                s = INFINITY;
                err |= ERR_NONFINITE;
            }
        }
        s = warp_max<float>(s);
        if ((threadIdx.x & 31) == 0 && s > 0.f) {
            const unsigned long long bits = (unsigned long long)__double_as_longlong((double)s);
            atomicMax(&b.st[i].amax_bits[b.parity], bits);
        }
        if (err) atomicOr(&b.st[i].err, err);
    }
}

// Host layout (per instance [cell][var][k] of u_kx, instances back to back in
// the order of the instance table) <-> group planes, one thread per cell.
// One cell (all variables) of a group's planes <-> its host-layout DOFs q
// ([var][k]), with the conversions of wcc_convert.cuh.
template <int K>
__device__ __forceinline__ void convert_cell(double* q, float* pl, long long pitch, long long c, int nv,
                                             int to_planes) {
    constexpr int NP = K + 1;
    for (int v = 0; v < nv; ++v) {
        float* p = pl + (long long)(v * NP) * pitch + c;
        float e[K];
        if (to_planes) {
            const ff u = host_to_mixed<K>(reinterpret_cast<const unsigned long long*>(q) + v * K, e);
            p[0] = u.hi;
            p[pitch] = u.lo;
#pragma unroll
            for (int k = 1; k < K; ++k) p[(long long)(k + 1) * pitch] = e[k];
        } else {
#pragma unroll
            for (int k = 1; k < K; ++k) e[k] = p[(long long)(k + 1) * pitch];
            mixed_to_host<K>(ff{p[0], p[pitch]}, e, reinterpret_cast<unsigned long long*>(q) + v * K);
        }
    }
}

template <int SYS, int PA, int PB>
__global__ void __launch_bounds__(kThreads) batch_convert(const BatchArgs b, double* aos, int to_planes) {
    for (long long tile = blockIdx.x; tile < b.total_tiles; tile += gridDim.x) {
        const int i = __ldg(b.tile_inst + tile);
        const BatchInstance I = b.inst[i];
        const long long c = (tile - b.tile_start[i]) * kTile + threadIdx.x;
        if (threadIdx.x >= kTile || c >= I.cells[b.parity]) continue;
        const int P = I.group == 0 ? PA : PB;
        const int K = P + 1, NV = nvars(SYS);
        float* pl = (to_planes ? b.out[I.group] : const_cast<float*>(b.in[I.group])) + I.offset;
        const long long pitch = b.pitch[I.group];
        double* q0 = aos + I.aos_offset[b.parity] + c * NV * K;
        if (I.group == 0)
            convert_cell<PA + 1>(q0, pl, pitch, c, NV, to_planes);
        else
            convert_cell<PB + 1>(q0, pl, pitch, c, NV, to_planes);
    }
}

}  // namespace wcc
