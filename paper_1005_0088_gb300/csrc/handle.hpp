// Internal state behind the C-ABI handles (ndsi_plan, ndsi_factors) and the helpers the entry
// points share: error reporting, device tables, workspaces, the schedule runner, the density
// sweep and the density-of-states sweep.
#pragma once

#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <memory>
#include <new>
#include <string>
#include <vector>

#include "kernels.cuh"
#include "ndsi.h"
#include "plan.hpp"
#include "split_gemm.cuh"
#include "solve.cuh"

namespace ndsi {
// Event-timed launch records, resolved after the stream synchronises, keyed by kernel family
// and schedule step ("gemm_split:schur", "diaginv", ...).
struct ProfStat {
    int64_t launches = 0;
    double ms = 0, flops = 0, bytes = 0, tensor_flops = 0;
};
struct ProfRec {
    int key;
    double flops, bytes, tensor_flops;
    cudaEvent_t e0, e1;
    int64_t launch;  // schedule launch index, or -1
};
struct Profiler {
    bool on = false;
    bool by_level = false;                  // family names carry the tree level (":L<level>")
    int64_t cur_launch = -1;                // schedule launch being issued (run_phase)
    std::vector<double>* per_launch = nullptr;  // when set: ms accumulated per launch index
    std::vector<cudaEvent_t> pool;
    size_t used = 0;
    std::vector<ProfRec> pending;
    std::vector<std::string> names;
    std::vector<ProfStat> stats;
    int key(const std::string& name) {
        for (size_t i = 0; i < names.size(); ++i)
            if (names[i] == name) return static_cast<int>(i);
        names.push_back(name);
        stats.emplace_back();
        return static_cast<int>(names.size()) - 1;
    }
};

// Split-precision metadata of a plan (built when opt.precision == NDSI_PREC_SPLIT).
struct SplitPlan {
    std::vector<SplitItem> items;
    std::vector<SplitStep> steps;
    std::vector<GemmTile> tiles;
    std::vector<SliceBlock> blocks;
    std::vector<int32_t> step_of_launch;
    std::vector<double> tensor_flops;   // per step, one pole
    std::vector<double> slice_bytes;    // per step, one pole: FP64 operand reads + BF16 slice writes
    std::vector<char> use_split;        // per launch: 1 = tensor-core path (autotuner may clear)
    std::vector<int8_t> bands;          // per launch: accumulator layout (0 per scale, 4 or 5 bands)
    int64_t generation = 0;             // bumped whenever the schedule is rebuilt
    SplitItem* d_items = nullptr;
    GemmTile* d_tiles = nullptr;
    SliceBlock* d_blocks = nullptr;
    void* blob = nullptr;
};
}  // namespace ndsi

struct ndsi_plan {
    ndsi::Plan P;
    ndsi::Profiler prof;
    ndsi::SplitPlan SP;
    ndsi::SplitBuffers SB;       // slice buffers of the density workspace
    ndsi::DevTables T;
    int device = -1;
    // density workspace (reused across calls)
    ndsi::Workspace W;
    double2* cw = nullptr;       // per-chunk points and weights
    double2* zw = nullptr;
    double2* cew = nullptr;      // energy-density weights of the same points
    unsigned long long* gersh = nullptr;  // Gershgorin bound of (H, S) for the moment points
    int32_t cw_cap = 0;
    double* partials = nullptr;  // trace reduction scratch
    double* dos_part = nullptr;  // per-point trace partials of the retarded-Green-function step
    double* dos_tr = nullptr;
    double2* dos_z = nullptr;
    int64_t dos_cap = 0;       // points (systems x energies)
    int64_t dos_part_cap = 0;  // doubles of dos_part
    double* stage = nullptr;     // staging for host H, S, rho, n_elec
    int64_t stage_cap = 0;
    std::vector<double> pole_z, pole_R;  // cached continued-fraction poles
    int32_t pole_M = 0;
    // CUDA graph of one density sweep (every chunk's factor, selected inversion and residue
    // sum), captured on first use and replayed while the buffers it names stay the same
    bool graphs = true;
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t graph = nullptr;
    std::vector<const void*> graph_key;
    int64_t graph_nodes = 0;
    double2* pin = nullptr;         // pinned staging of the point tables (3 x pin_cap)
    size_t pin_cap = 0;
    cudaEvent_t pin_ev = nullptr;   // recorded after the last copies out of `pin`
    // tables of the triangular solves (built on first use)
    ndsi::SolveTables ST;
    double2* point_z = nullptr;  // the single point factored for the eigensolver
};

struct ndsi_factors {
    ndsi_plan* plan = nullptr;
    ndsi::Workspace W;
    ndsi::SplitBuffers SB;
    double2* zd = nullptr;
    int32_t np = 0;
    bool inverted = false;  // ndsi_selinv has replaced the factors by G
    int64_t split_gen = 0;  // split schedule generation the factors were made with
    double2* solve_buf = nullptr;  // work space of ndsi_factors_solve (two n x k blocks)
    int64_t solve_cap = 0;         // complex elements per block
};

namespace ndsi {

// Record `msg` as the thread's last error and return `code`.
int fail(int code, const std::string& msg);

#define NDSI_CK(call)                                                                          \
    do {                                                                                       \
        cudaError_t e_ = (call);                                                               \
        if (e_ != cudaSuccess) {                                                               \
            return fail(e_ == cudaErrorMemoryAllocation ? NDSI_ERR_OOM : NDSI_ERR_CUDA,        \
                        std::string(#call) + ": " + cudaGetErrorString(e_));                   \
        }                                                                                      \
    } while (0)

template <class T>
inline size_t bytes_of(const std::vector<T>& v) {
    return v.size() * sizeof(T);
}

inline size_t align256(size_t x) { return (x + 255) & ~static_cast<size_t>(255); }

// Plan tables and workspaces.
int upload_tables(ndsi_plan* h);
bool is_device_ptr(const void* p);
bool foreign_device_ptr(const void* p);
int alloc_workspace(Workspace& W, const Plan& P, int32_t np);
void free_workspace(Workspace& W);
int64_t bytes_per_pole(const ndsi_plan* h);
int64_t workspace_cap(const ndsi_plan* h);
int ensure_stage(ndsi_plan* h, int64_t doubles);
// H, S on the device (host inputs are staged); the device status word after a sweep.
int device_inputs(ndsi_plan* h, const double* H, const double* S, const double** Hd, const double** Sd,
                  cudaStream_t st);
int check_status(ndsi_plan* h, cudaStream_t st);
// Every launch of one phase (0 factor, 1 selected inversion) for np points of z (stride zstride
// per system).
int run_phase(ndsi_plan* h, const Workspace& W, const SplitBuffers& SB, int phase, const double* H,
              const double* S, const double2* z, int64_t zstride, int np, cudaStream_t st, int slices = 0);
// Subset of the contour points of Eq. 8 a call sums: the poles begin <= p < end and, when m0 is
// set, the zeroth-moment point (all of them by default).
struct PoleRange {
    int32_t begin = 0, end = -1;
    bool m0 = true;
};
// rho (and e) and the per-system electron counts at per-system mu and kT (Eq. 8); with a pole
// range only that part of the sum (single-system plans, no energy density).
int density_impl(ndsi_plan* h, const double* Hd, const double* Sd, const double* mu, const double* kT,
                 int32_t n_poles, double* rho_d, double* ne_d, cudaStream_t st, double* e_d = nullptr,
                 const PoleRange* range = nullptr);
// Density of states (Eq. 41) of every system on its own grid, and of a single-system plan.
int dos_sweep_systems(ndsi_plan* h, const double* Hd, const double* Sd, const double* E, int nE, const double* eta,
                      double* D, cudaStream_t st);
int dos_sweep(ndsi_plan* h, const double* Hd, const double* Sd, const double* E, int nE, double eta, double* D,
              cudaStream_t st);

// (Re)build the split schedule of a plan from SplitPlan::bands; when its tables are on the device
// they are uploaded again and the slice buffers (whose tensor maps follow the schedule) dropped.
int rebuild_split(ndsi_plan* h);

// Measured FP64 (DFMA) throughput of the current device in TFLOP/s (peak.cu).
int fp64_rate(cudaStream_t st, double* tflops_out);

// Device buffer that frees itself (scratch of the solve and eigensolver entry points).
struct DevBuf {
    void* p = nullptr;
    ~DevBuf() {
        if (p) cudaFree(p);
    }
    template <class T>
    T* as() const {
        return static_cast<T*>(p);
    }
    cudaError_t alloc(size_t bytes) { return cudaMalloc(&p, std::max<size_t>(bytes, 16)); }
};

}  // namespace ndsi
