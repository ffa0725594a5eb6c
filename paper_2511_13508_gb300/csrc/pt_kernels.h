// pt_kernels.h -- parameter blocks and launchers of the device kernels (internal to the library).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>
#include "pt_common.cuh"

namespace ptgb {

struct SweepParams {
    const SampleDev *samples;
    const GroupDev *groups;
    int n_groups;
    const void *J;              // blocked J store (float or double)
    const int *bo;              // per sample: first block of each s-tile (ST+1)
    const int *xtlo;            // per sample: first x-tile of each s-tile (ST)
    const uint32_t *blkinfo;    // per sample block: (st << 16) | xt
    const int *mode_blk;        // per sample mode: block offset of the mode's run in the J store (N+1)
    void *a;                    // chain amplitudes (float2 or double2), chain-major
    double *E;                  // running energies per chain slot
    const int *label;           // chain slot -> temperature index
    const double *beta;         // temperature index -> beta
    unsigned long long *mc_acc; // per chain slot accepted moves
    unsigned long long *mc_att; // per chain slot attempted moves
    int R, nT, maxN;
    uint64_t seed;
    double cc;
    Control *ctl;
    int *progress;              // per group: runs written back in this launch
    int n_sweeps, sweeps_per_unit;
    int measure_every;          // snapshot at interior measurement points (0 = none)
    void *snap_a;               // [n_snap_max][a_total] complex
    double *snap_E;             // [n_snap_max][n_chains]
    int n_snap_max;
    int64_t a_total;            // complex numbers in one full state
    int n_chains;
    // update trace (armed by Control::trace_at / trace_update): [n_chains][kTraceRec] records, then the
    // pre-update states [a_total] as double complex, both in canonical (sample, replica, temperature) order
    double *trace;
    int nst;                    // coupling ring stages (set by the launcher)
};

struct FieldsParams {
    const SampleDev *samples;
    const GroupDev *groups;
    int group0;
    const void *J;
    const int *bo;
    const uint32_t *blkinfo;
    const int *mode_blk;
    const void *a;
    int j, k;
    double *out;  // [chains of sample][8]
};

struct EnergyParams {
    const SampleDev *samples;
    const GroupDev *groups;
    const void *J;
    const int *bo;
    const uint32_t *blkinfo;
    const int *mode_blk;
    const int *ebo;  // per sample mode: prefix count of blocks holding rows s > 2x (N+1)
    void *a;
    double cc;
    int renorm;
    double *E_out;   // optional: energies by chain slot
    double *E_state; // optional: running-energy array to overwrite
    Control *ctl;
    double *part;    // partial sums [group][part][32] (kEnergyPartsMax parts at most)
    int parts;       // thread blocks per group (1 .. kEnergyPartsMax)
};
constexpr int kEnergyPartsMax = 8;

// pt_sweep.cu
bool sweep_variant_exists(bool dbl, int G, int ncw);
cudaError_t launch_sweep(bool dbl, int G, int ncw, const SweepParams &p, int grid, cudaStream_t s);
int sweep_occupancy(bool dbl, int G, int ncw, int maxN);
cudaError_t launch_fields(bool dbl, int G, const FieldsParams &p, int ngroups, int maxN, cudaStream_t s);
cudaError_t launch_energy(bool dbl, int G, const EnergyParams &p, int ngroups, int maxN, cudaStream_t s);

// pt_aux.cu
struct InitParams {
    const SampleDev *samples;
    const int *chain_sample;  // chain slot -> sample
    const int *label;
    void *a;
    int dbl, R, nT;
    uint64_t seed;
};
cudaError_t launch_init(const InitParams &p, int n_chains, cudaStream_t s);

struct SwapParams {
    const SampleDev *samples;
    double *E;
    int *label;       // chain slot -> temperature index
    int *perm;        // [S][R][nT] temperature index -> chain slot
    const double *beta;
    unsigned long long *swap_acc, *swap_att;      // [S][R][nT-1]
    unsigned long long *mc_acc, *mc_att;          // per chain slot (folded here)
    unsigned long long *mcT_acc, *mcT_att;        // [S][nT]
    int S, R, nT;
    uint64_t seed;
    Control *ctl;
};
cudaError_t launch_swap(const SwapParams &p, cudaStream_t s);

struct MeasureParams {
    const SampleDev *samples;
    const void *a;          // live state
    const double *E;        // live energies
    const void *snap_a;     // snapshots
    const double *snap_E;
    int n_snap;             // snapshots to consume
    int live;               // also measure the live state
    const int *perm;        // [S][R][nT]
    int S, R, nT, dbl;
    int64_t a_total;
    int n_chains;
    double *stat;           // [S][nT][7]
    double *qstat;          // [S][nT][5]
    unsigned long long *qhist;  // [S][nT][201]
    unsigned long long *mc_acc, *mc_att, *mcT_acc, *mcT_att;
    const int *label;
};
cudaError_t launch_measure(const MeasureParams &p, cudaStream_t s);

// Plain FP64 path: the paper's design restated (one block per chain, one thread per quadruplet term).
// pt_graph.cu: FP32 sweep / energy on explicit interaction lists (one block per group of 8 chains)
// Row stride (in float2) of the FP32 group kernels' amplitude table: the 8 chains, unpadded.  The incidence records
// hold partner modes as row offsets (mode x this).
constexpr int kGraphRowStride = 8;

struct GraphParams {
    const SampleDev *samples;
    const GroupDev *groups;
    const int4 *quads;       // quadruplets in term order, per sample at q_off (energy kernel)
    const double *Jd;        // FP64 couplings (energy kernel)
    const int *inc_off;      // per sample mode: offsets into the incidence records (N+1, at mode_off)
    int max_deg;             // largest number of records of one mode, over all samples
    // incidence records per mode (at inc_off): the other three modes A, B, C as row offsets (mode x
    // kGraphRowStride), ordered so that the record's field term is J a_A a_B conj(a_C); w = position of the
    // record's own mode | positions of A, B, C << 2, 4, 6
    const int4 *rec;
    const float *recJ;       // coupling of each incidence record
    float2 *a;
    double *E;
    const int *label;
    const double *beta;
    unsigned long long *mc_acc, *mc_att;
    int R, nT, maxN;
    uint64_t seed;
    double cc;
    Control *ctl;
    int n_sweeps, measure_every;
    float2 *snap_a;
    double *snap_E;
    int n_snap_max;
    int64_t a_total;
    int n_chains;
    int renorm;              // energy kernel: rescale to sum |a|^4 = N first
    double *E_out, *E_state; // energy kernel outputs (optional)
    double *trace;           // sweep kernel: update trace (as SweepParams::trace; the cross term in place of B, A)
};
cudaError_t launch_wait_probe(Control *ctl, unsigned long long limit_ns, cudaStream_t s);
cudaError_t launch_graph_sweep(const GraphParams &p, int n_groups, cudaStream_t s);
cudaError_t launch_graph_energy(const GraphParams &p, int n_groups, cudaStream_t s);
cudaError_t graph_prepare(int maxN, int max_deg);  // shared-memory limits of the graph kernels (N <= maxN)

struct PlainParams {
    const SampleDev *samples;
    const int *chain_sample;
    const int4 *quads;       // canonical quadruplets of every sample
    const double *Jq;        // couplings, canonical order
    const int *inc_off;      // per sample mode: offsets into inc (N+1, at mode_off)
    const int *inc;          // per mode: quadruplet indices (sample-local) holding the mode
    double2 *a;
    double *E;
    const int *label;
    const double *beta;
    unsigned long long *mc_acc, *mc_att;
    int R, nT, maxN;
    uint64_t seed;
    double cc;
    Control *ctl;
    int n_sweeps, measure_every;
    double2 *snap_a;
    double *snap_E;
    int n_snap_max;
    int64_t a_total;
    int n_chains;
    int renorm;              // energy kernel: rescale first
    int write_state;         // energy kernel: overwrite the running energies
    double *E_out;
};
cudaError_t launch_plain_sweep(const PlainParams &p, int n_chains, cudaStream_t s);
cudaError_t launch_plain_energy(const PlainParams &p, int n_chains, cudaStream_t s);

cudaError_t launch_advance(Control *ctl, long long sweeps, long long swap_passes, long long rounds, cudaStream_t s);

}  // namespace ptgb
