// Serial level-by-level LoD selection on the GPU: the comparison baseline of
// §3.2 (Eq. 3, the LoG-style hierarchical filtering the paper replaces).
//
// Starting from the root, each level is one kernel over the current frontier:
// a node that passes R&L is selected; otherwise its children join the next
// frontier (an internal node out of the frustum does not prune its subtree, as
// in the per-node filter).  The host reads the next frontier's size after every
// level to size the following launch: one launch and one synchronisation per
// level, the T_synch term of Eq. 3.  The selected set equals the traversal-free
// filter's; it is written as bits and compacted by the same compaction kernel.
#include "fgs_internal.cuh"

namespace fgs {

__global__ void __launch_bounds__(256) levelwise_step_kernel(
    DevTree t, DevCamera cam, const uint32_t* __restrict__ child_start,
    const uint32_t* __restrict__ children, const uint32_t* __restrict__ frontier, uint32_t n_front,
    uint32_t* __restrict__ next, uint32_t* __restrict__ n_next, uint32_t* __restrict__ selbits)
{
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t lane = threadIdx.x & 31;
    uint32_t n = 0, c0 = 0, nc = 0;
    bool pass = false;
    if (i < n_front) {
        n = __ldg(frontier + i);
        const size_t np = t.n_pad;
        float vx, vy, vz, txtz = 0.0f, tytz = 0.0f;
        camera_space(cam, __ldg(t.mu + n), __ldg(t.mu + np + n), __ldg(t.mu + 2 * np + n), vx, vy, vz);
        const bool inf = frustum_test(cam, vx, vy, vz, txtz, tytz);
        const bool leaf = (__ldg(t.leaf_bits + (n >> 5)) >> (n & 31)) & 1u;
        if (inf) {
            if (leaf) {
                pass = true;
            } else {
                float s6[6];
#pragma unroll
                for (int q = 0; q < 6; ++q) s6[q] = __ldg(t.cov + q * np + n);
                float a, b, c, lam;
                ewa_cov2d(cam, vz, txtz, tytz, s6, a, b, c, lam);
                pass = fm(3.0f, fsq(lam)) <= cam.tau_R;
            }
        }
        if (pass) {
            atomicOr(selbits + (n >> 5), 1u << (n & 31));
        } else {
            c0 = __ldg(child_start + n);
            nc = __ldg(child_start + n + 1) - c0;
        }
    }
    // warp-aggregated append of the children of the nodes that did not pass
    uint32_t incl = nc;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t up = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= (uint32_t)o) incl += up;
    }
    const uint32_t wtot = __shfl_sync(0xffffffffu, incl, 31);
    uint32_t base = 0;
    if (lane == 31 && wtot) base = atomicAdd(n_next, wtot);
    base = __shfl_sync(0xffffffffu, base, 31);
    const uint32_t first = base + incl - nc;
    for (uint32_t k = 0; k < nc; ++k) next[first + k] = __ldg(children + c0 + k);
}

void launch_levelwise_step(const DevTree& t, const DevCamera& cam, const uint32_t* child_start,
                           const uint32_t* children, const uint32_t* frontier, uint32_t n_front,
                           uint32_t* next, uint32_t* n_next, uint32_t* selbits, cudaStream_t s)
{
    const unsigned blocks = (n_front + 255) / 256;
    levelwise_step_kernel<<<blocks, 256, 0, s>>>(t, cam, child_start, children, frontier, n_front,
                                                 next, n_next, selbits);
}

}  // namespace fgs
