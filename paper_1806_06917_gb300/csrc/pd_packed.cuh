// pd_packed.cuh -- the request server's packed kernel: every active request of
// the server advanced by one explicit step in one launch ("round"), its CTAs
// taking (request, pass, tile) work items from a device-side list.
//
// Work items of round s (the s-th step of the quantum): for every request with
// more than s steps left in the quantum, group A holds one item per tile for
// its first pass (the fused PMB force + update, or the LPS dilatation) and
// group B one per tile for the LPS force + update pass; A comes first. An LPS
// force item needs the dilatation of its 27 neighbour tiles (theta of the halo),
// which items of group A of the same launch compute: its CTA waits for their
// completion flags, a bounded wait that ends the launch with an error status
// after a time limit instead of hanging. Items are claimed in list order and a
// claimed item's CTA stays resident until it is done, so every item waited on
// is already held by a running CTA: the waits end.
#pragma once

#include "pd_tile.cuh"

struct pd_sim;

namespace pdk {

enum PackKind { PK_PMB3 = 0, PK_PMB2 = 1, PK_LPS = 2 };

constexpr int PACK_THREADS = 512;         // CTA size: the LPS force pass of a 2^9-point tile

// The LPS passes' stencil tables (3 float4 per stencil entry, the dilatation's
// then the force pass's) for horizons m = 1, 2, 3 on 2^9-point (8 x 8 x 8)
// tiles, carried in the kernel's parameter bank (read as constant-bank loads,
// as the simulations' own kernels read theirs) instead of shared memory: they
// depend on m alone. Stencil sizes 6, 32 and 122.
constexpr int PACK_LPS_MMAX = 3;
constexpr int PACK_TAB_N = 2 * 3 * (6 + 32 + 122);
inline int pack_lps_stencil(int m) { return m == 1 ? 6 : m == 2 ? 32 : m == 3 ? 122 : 0; }
// Offset of horizon m's dilatation table (which = 0) or force table (which = 1).
inline int pack_tab_offset(int m, int which)
{
    int off = 0;
    for (int k = 1; k < m; ++k) off += 2 * 3 * pack_lps_stencil(k);
    return off + which * 3 * pack_lps_stencil(m);
}

// One request of a quantum (device table entry, built by the server).
struct PackReq {
    TileArgs a[2];          // MODE_STEP arguments by staging parity (src = hl[p], dst = hl[p ^ 1]),
                            // with the flags of every step after the quantum's first
    int kind;               // PackKind
    int split;              // PMB: threads per point pair of its body (1 or 2)
    int ntiles;
    int nsteps;             // rounds this request takes part in
    int cur0;               // staging parity at the quantum's start
    int vhalf0, cd0;        // v_is_half and the central-difference flag of the quantum's first step
    int tab_dil, tab_force; // LPS: offsets of its tables in PackTable.tabs
    int pad_;
    unsigned *dil_done;     // LPS: per tile, 1 + the step of its last dilatation (monotonic)
    long long step0;        // the simulation's step count at the quantum's start
};

// Status word of a quantum (device): code, request, tile, round of the first failure.
enum { PACK_OK = 0, PACK_TIMEOUT = 1 };

// Kernel parameters of a quantum's rounds.
struct PackTable {
    const PackReq *req;     // sorted by nsteps, descending
    const int *offA;        // [nreq + 1] prefix sums of the requests' group-A items
    const int *offB;        // [nreq + 1] the same for group B
    const int *nsteps;      // [nreq] req[r].nsteps (descending)
    unsigned *counters;     // [rounds] item counters, zero at the quantum's start
    unsigned *status;       // [4]
    long long wait_ns;      // limit of one wait
    int nreq;
    int stall;              // tests only: the first group-B item of round 0 waits on a flag nothing sets
    float4 tabs[PACK_TAB_N];  // the LPS tables (pack_tab_offset)
};

// What the server needs of a simulation to pack it (pd_api.cu).
struct PackInfo {
    int eligible;           // the packed kernel can step it (FP32C, PMB without breaking or LPS without
                            // partial volume and m <= 3, 2^9-point tiles, pair_threads as the packed body's)
    int kind, split, ntiles;
    int m;                  // horizon in lattice spacings
    const float4 *htab_dil, *htab_force;   // LPS: the simulation's host tables (3 pack_lps_stencil(m) float4 each)
    size_t smem;
    TileArgs a[2];          // MODE_STEP by staging parity, flags of a step after the first
    int cur, vhalf, cd0, cd;
    long long step;
};
int sim_pack_info(pd_sim *s, PackInfo *pi);
// Bookkeeping after n packed steps (staging parity, step count, half-step velocity).
void sim_pack_advance(pd_sim *s, long long n);
// The packed body's threads per point pair for a lattice: 2 where the stencil
// has at least two 32-bond words (all PACK_THREADS threads busy), else 1.
inline int pack_split_for(int W) { return W >= 2 ? 2 : 1; }

// Host side (pd_packed.cu). Dynamic shared memory of a request's items, and the
// resident CTAs per SM of the kernel at that size.
size_t pack_smem(const Geom &g, int kind, int split);
int pack_occupancy(size_t smem, int *ctas_per_sm);
// Enqueue `rounds` rounds (round indices 0 .. rounds - 1) on st with `grid` CTAs.
int pack_launch_rounds(const PackTable &t, int rounds, int grid, size_t smem, cudaStream_t st);

}  // namespace pdk
