// Projection, SH colour and scene-adaptive shrinking (§3.1, §3.3) on sm_103a.
//
// project_kernel: one thread per selected Gaussian computes the splat record
// (centre, conic, log-domain skip threshold, opacity, depth, colour, footprint
// radius) and its footprint record (tile rectangle, pair count, depth bits);
// then each warp enumerates its Gaussians' Gaussian-tile pairs and counts them
// into their tiles, from which the tile ranges of the sorted pair list follow
// (pairs.cu); the pairs of a Gaussian with more than kWarpWidePairs of them
// are counted by all the warp's lanes at once.
#include "pairs_impl.cuh"
#include "project_impl.cuh"

namespace fgs {

__global__ void __launch_bounds__(kProjThreads) project_kernel(
    DevTree t, DevCamera cam, const uint32_t* __restrict__ sel, float* __restrict__ splat,
    uint4* __restrict__ foot, uint32_t* __restrict__ tile_cnt, FrameState* st)
{
    grid_dep_wait();
    grid_dep_trigger();
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t M = st->M;
    const uint32_t n_groups = (M + kProjThreads - 1) / kProjThreads;
    for (uint32_t g = blockIdx.x; g < n_groups; g += gridDim.x) {
        const uint32_t m = g * kProjThreads + threadIdx.x;
        uint4 f = make_uint4(0, 0, 0, 0);
        if (m < M) f = proj::project_one(t, cam, __ldg(sel + m), m, splat, foot);
        const uint32_t emitting = __popc(__ballot_sync(0xffffffffu, f.z > 0));
        if (lane == 0 && emitting) atomicAdd(&st->n_emitting, emitting);
        warp_count_pairs(f.z, f.x, f.y, (uint32_t)cam.tiles_x, 0u, tile_cnt);
    }
}

void launch_project(const DevTree& t, const DevCamera& cam, const uint32_t* sel, float* splat,
                    uint4* foot, uint32_t* tile_cnt, FrameState* st, int blocks, cudaStream_t s)
{
    if (blocks < 1) blocks = 1;
    launch_pdl(project_kernel, blocks, kProjThreads, 0, s, t, cam, sel, splat, foot, tile_cnt, st);
}

int occ_project()
{
    int b = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, project_kernel, kProjThreads, 0);
    return b > 0 ? b : 1;
}

}  // namespace fgs
