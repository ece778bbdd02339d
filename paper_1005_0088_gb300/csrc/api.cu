// C-ABI entry points: plan life cycle, pole-batched factor / selected inversion / density.
#include "handle.hpp"

namespace ndsi {

namespace {
thread_local std::string g_last_error;
}

void set_last_error(const std::string& msg) { g_last_error = msg; }

int fail(int code, const std::string& msg) {
    set_last_error(msg);
    return code;
}

// Upload every index table of the plan into one device allocation (first use only).
static int upload_split(ndsi_plan* h);

int upload_tables(ndsi_plan* h) {
    if (h->T.blob) return NDSI_OK;
    Plan& P = h->P;
    NDSI_CK(cudaGetDevice(&h->device));
    struct Part {
        const void* src;
        size_t bytes;
        void** dst;
    };
    DevTables& T = h->T;
    std::vector<Part> parts = {
        {P.nodes.data(), bytes_of(P.nodes), reinterpret_cast<void**>(&T.nodes)},
        {P.asm_map.data(), bytes_of(P.asm_map), reinterpret_cast<void**>(&T.asm_map)},
        {P.out_map.data(), bytes_of(P.out_map), reinterpret_cast<void**>(&T.out_map)},
        {P.inv_map.data(), bytes_of(P.inv_map), reinterpret_cast<void**>(&T.inv_map)},
        {P.rel_map.data(), bytes_of(P.rel_map), reinterpret_cast<void**>(&T.rel_map)},
        {P.scatter_idx.data(), bytes_of(P.scatter_idx), reinterpret_cast<void**>(&T.scatter_idx)},
        {P.gemm_items.data(), bytes_of(P.gemm_items), reinterpret_cast<void**>(&T.gemm_items)},
        {P.gemm_tiles.data(), bytes_of(P.gemm_tiles), reinterpret_cast<void**>(&T.gemm_tiles)},
        {P.copy_items.data(), bytes_of(P.copy_items), reinterpret_cast<void**>(&T.copy_items)},
        {P.diag_items.data(), bytes_of(P.diag_items), reinterpret_cast<void**>(&T.diag_items)},
        {P.node_tiles.data(), bytes_of(P.node_tiles), reinterpret_cast<void**>(&T.node_tiles)},
        {P.entry_sys.data(), bytes_of(P.entry_sys), reinterpret_cast<void**>(&T.entry_sys)},
        {P.rowptr.data(), bytes_of(P.rowptr), reinterpret_cast<void**>(&T.rowptr)},
        {P.col.data(), bytes_of(P.col), reinterpret_cast<void**>(&T.col)},
        {nullptr, sizeof(int) * 4, reinterpret_cast<void**>(&T.status)},
    };
    size_t total = 0;
    for (const Part& p : parts) total += align256(std::max<size_t>(p.bytes, 16));
    void* blob = nullptr;
    NDSI_CK(cudaMalloc(&blob, total));
    T.blob = blob;
    size_t off = 0;
    for (const Part& p : parts) {
        char* dst = static_cast<char*>(blob) + off;
        *p.dst = dst;
        if (p.src && p.bytes) NDSI_CK(cudaMemcpy(dst, p.src, p.bytes, cudaMemcpyHostToDevice));
        off += align256(std::max<size_t>(p.bytes, 16));
    }
    NDSI_CK(cudaMemset(T.status, 0, sizeof(int) * 4));
    NDSI_CK(kernels_init());
    if (P.opt.precision == NDSI_PREC_SPLIT) {
        int rc = upload_split(h);
        if (rc) return rc;
        NDSI_CK(split_init());
    }
    return NDSI_OK;
}

bool is_device_ptr(const void* p) {
    if (!p) return false;
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Device memory of a GPU other than the current one: the kernels cannot use it (and staging
// it as host memory would be wrong too), so the entry points refuse it.
bool foreign_device_ptr(const void* p) {
    if (!p) return false;
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice && a.device != dev;
}

int alloc_workspace(Workspace& W, const Plan& P, int32_t np) {
    if (W.np_cap >= np && W.fronts) return NDSI_OK;
    if (W.fronts) cudaFree(W.fronts);
    if (W.scr) cudaFree(W.scr);
    W = Workspace{};
    W.front_stride = P.front_total;
    W.scr_stride = P.scr_total;
    NDSI_CK(cudaMalloc(&W.fronts, sizeof(double2) * static_cast<size_t>(W.front_stride) * np));
    NDSI_CK(cudaMalloc(&W.scr, sizeof(double2) * static_cast<size_t>(W.scr_stride) * np));
    W.np_cap = np;
    return NDSI_OK;
}

void free_workspace(Workspace& W) {
    if (W.fronts) cudaFree(W.fronts);
    if (W.scr) cudaFree(W.scr);
    W = Workspace{};
}

const char* tag_name(int tag) {
    static const char* const names[] = {"assemble", "scatter", "dinv",  "panel",    "update",  "pcopy",
                                        "ainv_t",   "ainv_d",  "ainv_copy", "lrj",   "schur",   "lcopy",
                                        "gather",   "sel_t",   "sel_d",   "sel_copy", "opanel",  "oupdate",
                                        "opcopy",   "oainv_t", "oainv_d", "oainv_copy"};
    constexpr int n = static_cast<int>(sizeof(names) / sizeof(names[0]));
    return (tag >= 0 && tag < n) ? names[tag] : "other";
}

std::string family_of(const Launch& l) {
    switch (l.kind) {
        case L_GEMM: return std::string("gemm_f64:") + tag_name(l.tag);
        case L_DIAGINV: return "diaginv";
        case L_ASSEMBLE: return "assemble";
        case L_SCATTER: return "scatter";
        case L_COPY: return "copy";
        case L_GATHER: return "gather";
        default: return "other";
    }
}

cudaEvent_t prof_event(Profiler& pf) {
    if (pf.used == pf.pool.size()) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        pf.pool.push_back(e);
    }
    return pf.pool[pf.used++];
}

// Bracket a launch with events when profiling; `fn` performs the launch.
template <class Fn>
cudaError_t timed(Profiler& pf, const std::string& family, double flops, double bytes, cudaStream_t st, Fn fn,
                  double tensor_flops = 0) {
    if (!pf.on) return fn();
    cudaEvent_t e0 = prof_event(pf), e1 = prof_event(pf);
    if (e0) cudaEventRecord(e0, st);
    cudaError_t e = fn();
    if (e1) cudaEventRecord(e1, st);
    if (e0 && e1) pf.pending.push_back(ProfRec{pf.key(family), flops, bytes, tensor_flops, e0, e1, pf.cur_launch});
    return e;
}

// Fold finished records into the per-family totals (the stream has been synchronised).
void prof_resolve(Profiler& pf) {
    for (const ProfRec& r : pf.pending) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, r.e0, r.e1) == cudaSuccess) {
            ProfStat& st = pf.stats[r.key];
            st.ms += ms;
            st.flops += r.flops;
            st.bytes += r.bytes;
            st.tensor_flops += r.tensor_flops;
            st.launches += 1;
            if (pf.per_launch && r.launch >= 0 && r.launch < static_cast<int64_t>(pf.per_launch->size()))
                (*pf.per_launch)[r.launch] += ms;
        } else {
            cudaGetLastError();
        }
    }
    pf.pending.clear();
    pf.used = 0;
}

int run_phase(ndsi_plan* h, const Workspace& W, const SplitBuffers& SB, int phase, const double* H,
              const double* S, const double2* z, int64_t zstride, int np, cudaStream_t st, int slices) {
    const Plan& P = h->P;
    const bool split = P.opt.precision == NDSI_PREC_SPLIT;
    // digits per operand of this batch of points (the slice buffers keep the layout of
    // opt.split_slices; a smaller count fills and reads only the leading digits)
    const int ns = slices > 0 ? slices : P.opt.split_slices;
    const double pair_frac = split ? static_cast<double>(ns * (ns + 1)) / (P.opt.split_slices * (P.opt.split_slices + 1)) : 1.0;
    for (size_t li = 0; li < P.launches.size(); ++li) {
        const Launch& l = P.launches[li];
        if (l.phase != phase) continue;
        cudaError_t e;
        h->prof.cur_launch = static_cast<int64_t>(li);
        if (split && split_eligible(l) && h->SP.use_split[li]) {
            const int si = h->SP.steps.empty() ? 0 : h->SP.step_of_launch[li];
            const SplitStep& step = h->SP.steps[si];
            const double2* bufs[2] = {W.fronts, W.scr};
            const int64_t strides[2] = {W.front_stride, W.scr_stride};
            const std::string tg = std::string(tag_name(l.tag)) +
                                   (h->prof.by_level ? ":L" + std::to_string(l.level) : std::string());
            e = timed(h->prof, "slice:" + tg, 0.0, h->SP.slice_bytes[si] * np, st, [&]() {
                return split_slice_step(l, h->T.gemm_items, h->SP.d_items, h->SP.d_blocks, step, SB, ns,
                                        bufs[l.bufA], strides[l.bufA], bufs[l.bufB], strides[l.bufB], np, st);
            });
            if (e == cudaSuccess)
                e = timed(
                    h->prof, "gemm_split:" + tg, l.flops * np, l.bytes * np, st,
                    [&]() {
                        return split_mma_step(l, si, h->T.gemm_items, h->SP.d_items, h->SP.d_tiles, step, SB, ns,
                                              const_cast<double2*>(bufs[l.bufC]), strides[l.bufC], np,
                                              h->T.status, st);
                    },
                    h->SP.tensor_flops[si] * np * pair_frac);
        } else {
            e = timed(h->prof,
                      family_of(l) + (h->prof.by_level && l.kind == L_GEMM ? ":L" + std::to_string(l.level) : std::string()),
                      l.flops * np, l.bytes * np, st,
                      [&]() { return launch_step(P, h->T, l, W, H, S, z, zstride, np, st); });
        }
        if (e != cudaSuccess)
            return fail(NDSI_ERR_CUDA, std::string("kernel launch (step ") + std::to_string(l.tag) +
                                           "): " + cudaGetErrorString(e));
    }
    return NDSI_OK;
}

int check_status(ndsi_plan* h, cudaStream_t st) {
    int hs[4] = {0, 0, 0, 0};
    NDSI_CK(cudaMemcpyAsync(hs, h->T.status, sizeof(hs), cudaMemcpyDeviceToHost, st));
    NDSI_CK(cudaStreamSynchronize(st));
    prof_resolve(h->prof);
    if (hs[0] != 0) {
        NDSI_CK(cudaMemsetAsync(h->T.status, 0, sizeof(int) * 4, st));
        NDSI_CK(cudaStreamSynchronize(st));
        if (hs[0] & kStatusBadItem) return fail(NDSI_ERR_INVALID, "internal: a diagonal block wider than its kernel");
        if (hs[0] & kStatusSingular) return fail(NDSI_ERR_SINGULAR, "singular or non-finite pivot block");
        return fail(NDSI_ERR_TIMEOUT, "bounded device wait gave up");
    }
    return NDSI_OK;
}

int ensure_stage(ndsi_plan* h, int64_t doubles) {
    if (h->stage_cap >= doubles) return NDSI_OK;
    if (h->stage) cudaFree(h->stage);
    h->stage = nullptr;
    h->stage_cap = 0;
    NDSI_CK(cudaMalloc(&h->stage, sizeof(double) * static_cast<size_t>(doubles)));
    h->stage_cap = doubles;
    return NDSI_OK;
}

// Device copies of H and S (staged when the caller passed host memory).
int device_inputs(ndsi_plan* h, const double* H, const double* S, const double** Hd,
                  const double** Sd, cudaStream_t st) {
    const int64_t nnz = h->P.nnz;
    if (foreign_device_ptr(H) || foreign_device_ptr(S))
        return fail(NDSI_ERR_INVALID, "H or S is device memory of another GPU");
    const bool hd = is_device_ptr(H), sd = is_device_ptr(S);
    if (!hd || !sd) {
        int rc = ensure_stage(h, 3 * nnz + 8);
        if (rc) return rc;
    }
    *Hd = H;
    *Sd = S;
    if (!hd) {
        NDSI_CK(cudaMemcpyAsync(h->stage, H, sizeof(double) * nnz, cudaMemcpyHostToDevice, st));
        *Hd = h->stage;
    }
    if (!sd) {
        NDSI_CK(cudaMemcpyAsync(h->stage + nnz, S, sizeof(double) * nnz, cudaMemcpyHostToDevice, st));
        *Sd = h->stage + nnz;
    }
    return NDSI_OK;
}

// Device bytes one pole needs: fronts, scratch and (split mode) the largest step's slices.
int64_t bytes_per_pole(const ndsi_plan* h) {
    int64_t b = int64_t(16) * (h->P.front_total + h->P.scr_total);
    if (h->P.opt.precision == NDSI_PREC_SPLIT) {
        int64_t a = 0, bb = 0, ea = 0, eb = 0;
        for (const SplitStep& st : h->SP.steps) {
            a = std::max<int64_t>(a, st.rowsA * st.Kcols);
            bb = std::max<int64_t>(bb, st.rowsB * st.Kcols);
            ea = std::max<int64_t>(ea, st.erowsA);
            eb = std::max<int64_t>(eb, st.erowsB);
        }
        b += 2 * (a + bb) + 4 * (ea + eb);
    }
    return b;
}

int64_t workspace_cap(const ndsi_plan* h) {
    if (h->P.opt.max_workspace_bytes > 0) return h->P.opt.max_workspace_bytes;
    size_t freeb = 0, totalb = 0;
    if (cudaMemGetInfo(&freeb, &totalb) != cudaSuccess) {
        cudaGetLastError();
        return int64_t(8) << 30;
    }
    int64_t have = static_cast<int64_t>(freeb) + static_cast<int64_t>(h->W.np_cap) * bytes_per_pole(h);
    return static_cast<int64_t>(0.85 * static_cast<double>(have));
}

}  // namespace ndsi

namespace ndsi {
// Slice count of a split plan when the caller leaves it to the library: six BF16 digits (47
// bits).  A seventh changes nothing with four accumulator bands (the tail accumulator's floor
// dominates) and little with five.
int auto_slices(const Plan&) { return 6; }

// Accumulators when the caller leaves it to the library: one per slice-product scale (reported as
// 0 in the options, S in ndsi_plan_info).  The tail variants (4 or 5) mix the smallest scales in
// one accumulator, where the tensor core drops the low bits of the smaller products (a floor near
// 2^-38 or 2^-43 of the result); one accumulator per scale has no such floor, and because each A
// digit's products are one wide MMA the operand tiles are read from shared memory once per digit,
// which is what limited the tail variants' tensor throughput at N = 96.
int auto_bands(const Plan&) { return 0; }

// Split-precision metadata of a plan: tensor-core steps, their tile lists and cost figures.
static void build_split_metadata(ndsi_plan* h) {
    SplitPlan& S = h->SP;
    const int slices = h->P.opt.split_slices;
    build_split_schedule(h->P, slices, S.bands, S.items, S.steps, S.tiles, S.blocks);
    S.step_of_launch.assign(h->P.launches.size(), -1);
    S.tensor_flops.clear();
    S.slice_bytes.clear();
    int k = 0;
    for (size_t li = 0; li < h->P.launches.size(); ++li) {
        const Launch& l = h->P.launches[li];
        if (!split_eligible(l)) continue;
        const SplitStep& st = S.steps[k];
        S.tensor_flops.push_back(split_executed_flops(h->P, st, S.items, S.tiles, l, slices));
        double sb = 0;
        for (int64_t i = 0; i < l.count; ++i) {
            const GemmItem& g = h->P.gemm_items[l.first + i];
            // FP64 operand reads: once (one-pass slicer) or twice (two-pass)
            sb += (st.slice_ldt > 0 ? 1.0 : 2.0) * 16.0 * (static_cast<double>(g.M) * g.K + static_cast<double>(g.N) * g.K);
        }
        sb += 2.0 * (static_cast<double>(st.rowsA) + st.rowsB) * st.Kcols;
        S.slice_bytes.push_back(sb);
        S.step_of_launch[li] = k++;
    }
    ++S.generation;
}

void setup_split(ndsi_plan* h, const ndsi_options& o) {
    SplitPlan& S = h->SP;
    S.bands.assign(h->P.launches.size(), static_cast<int8_t>(o.split_bands));
    S.use_split.assign(h->P.launches.size(), 1);
    build_split_metadata(h);
}

static int upload_split(ndsi_plan* h) {
    SplitPlan& S = h->SP;
    if (S.blob) cudaFree(S.blob);
    S.blob = nullptr;
    const size_t bi = align256(std::max<size_t>(bytes_of(S.items), 16));
    const size_t bt = align256(std::max<size_t>(bytes_of(S.tiles), 16));
    const size_t bb = align256(std::max<size_t>(bytes_of(S.blocks), 16));
    NDSI_CK(cudaMalloc(&S.blob, bi + bt + bb));
    S.d_items = reinterpret_cast<SplitItem*>(S.blob);
    S.d_tiles = reinterpret_cast<GemmTile*>(static_cast<char*>(S.blob) + bi);
    S.d_blocks = reinterpret_cast<SliceBlock*>(static_cast<char*>(S.blob) + bi + bt);
    if (!S.items.empty()) NDSI_CK(cudaMemcpy(S.d_items, S.items.data(), bytes_of(S.items), cudaMemcpyHostToDevice));
    if (!S.tiles.empty()) NDSI_CK(cudaMemcpy(S.d_tiles, S.tiles.data(), bytes_of(S.tiles), cudaMemcpyHostToDevice));
    if (!S.blocks.empty()) NDSI_CK(cudaMemcpy(S.d_blocks, S.blocks.data(), bytes_of(S.blocks), cudaMemcpyHostToDevice));
    return NDSI_OK;
}

int rebuild_split(ndsi_plan* h) {
    NDSI_CK(cudaDeviceSynchronize());   // no launch of the old schedule may still read its tables
    build_split_metadata(h);
    split_free(h->SB);
    if (h->graph) {
        cudaGraphExecDestroy(h->graph);
        h->graph = nullptr;
        h->graph_key.clear();
        h->graph_nodes = 0;
    }
    return h->T.blob ? upload_split(h) : NDSI_OK;
}
int sweep(ndsi_plan* h, const double* Hd, const double* Sd, int32_t nq, int32_t n_near, int32_t chunk,
          const std::vector<int>& part_off, double* rho_d, double* ne_d, double* e_d, cudaStream_t st);

}  // namespace ndsi

using namespace ndsi;

extern "C" {

void ndsi_default_options(ndsi_options* opt) {
    if (!opt) return;
    opt->leaf_atoms = 20;
    opt->precision = NDSI_PREC_FP64;
    opt->split_slices = 0;
    opt->block = 16;
    opt->m0_radius = 1e7;
    opt->max_workspace_bytes = 0;
    opt->outer_block = 128;
    opt->split_bands = 0;
    opt->cell[0] = opt->cell[1] = opt->cell[2] = 0.0;
    opt->screen_degree = 0;
    opt->split_far_ratio = 0.0;
}

int ndsi_poles(int32_t M, double* z_out, double* R_out) {
    std::string err;
    int rc = cf_poles(M, z_out, R_out, err);
    if (rc) set_last_error(err);
    return rc;
}

int ndsi_analyze(const ndsi_pattern* pat, int32_t n_atoms, const double* centers,
                 const int32_t* atom_of_basis, const ndsi_options* opt, ndsi_plan** plan_out) {
    if (!plan_out) return fail(NDSI_ERR_INVALID, "ndsi_analyze: plan_out is NULL");
    *plan_out = nullptr;
    ndsi_options o;
    ndsi_default_options(&o);
    if (opt) o = *opt;
    if (o.m0_radius <= 0) o.m0_radius = 1e7;
    if (o.precision != NDSI_PREC_FP64 && o.precision != NDSI_PREC_SPLIT)
        return fail(NDSI_ERR_INVALID, "ndsi_analyze: unknown precision");
    ndsi_plan* h = new (std::nothrow) ndsi_plan();
    if (!h) return fail(NDSI_ERR_OOM, "ndsi_analyze: out of host memory");
    std::string err;
    int rc;
    try {
        rc = analyze(pat, n_atoms, centers, atom_of_basis, o, h->P, err);
    } catch (const std::bad_alloc&) {
        rc = NDSI_ERR_OOM;
        err = "ndsi_analyze: out of host memory";
    } catch (...) {
        rc = NDSI_ERR_INVALID;
        err = "ndsi_analyze: internal error";
    }
    if (rc) {
        delete h;
        return fail(rc, err);
    }
    if (o.precision == NDSI_PREC_SPLIT) {
        if (o.split_slices != 0 && (o.split_slices < 4 || o.split_slices > kSplitMaxSlices)) {
            delete h;
            return fail(NDSI_ERR_INVALID, "ndsi_analyze: split_slices must be 0 or in [4, 7]");
        }
        if (o.split_bands != 0 && o.split_bands != 4 && o.split_bands != 5) {
            delete h;
            return fail(NDSI_ERR_INVALID, "ndsi_analyze: split_bands must be 0, 4 or 5");
        }
        if (o.split_slices == 0) o.split_slices = auto_slices(h->P);
        if (o.split_bands == 0) o.split_bands = auto_bands(h->P);
        if (!std::isfinite(o.split_far_ratio) || (o.split_far_ratio > 0 && o.split_far_ratio < 1)) {
            delete h;
            return fail(NDSI_ERR_INVALID, "ndsi_analyze: split_far_ratio must be 0, negative or >= 1");
        }
        if (o.split_far_ratio == 0) o.split_far_ratio = kSplitFarRatio;
        h->P.opt.split_slices = o.split_slices;
        h->P.opt.split_bands = o.split_bands;
        h->P.opt.split_far_ratio = o.split_far_ratio;
        setup_split(h, o);
    }
    *plan_out = h;
    return NDSI_OK;
}

int ndsi_analyze_batched(int32_t n_systems, const ndsi_pattern* pats, const int32_t* n_atoms,
                         const double* const* centers, const int32_t* const* atom_of_basis,
                         const ndsi_options* opt, ndsi_plan** plan_out) {
    if (!plan_out || n_systems < 1 || !pats || !n_atoms || !centers || !atom_of_basis)
        return fail(NDSI_ERR_INVALID, "ndsi_analyze_batched: invalid argument");
    *plan_out = nullptr;
    ndsi_options o;
    ndsi_default_options(&o);
    if (opt) o = *opt;
    if (o.m0_radius <= 0) o.m0_radius = 1e7;
    std::vector<Plan> parts(n_systems);
    std::string err;
    try {
        for (int32_t i = 0; i < n_systems; ++i) {
            int rc = analyze(&pats[i], n_atoms[i], centers[i], atom_of_basis[i], o, parts[i], err);
            if (rc) return fail(rc, "system " + std::to_string(i) + ": " + err);
        }
        ndsi_plan* h = new ndsi_plan();
        int rc = merge_plans(parts, h->P, err);
        if (rc) {
            delete h;
            return fail(rc, err);
        }
        if (o.precision == NDSI_PREC_SPLIT) {
            if (o.split_slices != 0 && (o.split_slices < 4 || o.split_slices > kSplitMaxSlices)) {
                delete h;
                return fail(NDSI_ERR_INVALID, "ndsi_analyze_batched: split_slices must be 0 or in [4, 7]");
            }
            if (o.split_bands != 0 && o.split_bands != 4 && o.split_bands != 5) {
                delete h;
                return fail(NDSI_ERR_INVALID, "ndsi_analyze_batched: split_bands must be 0, 4 or 5");
            }
            if (o.split_slices == 0) o.split_slices = auto_slices(h->P);
            if (o.split_bands == 0) o.split_bands = auto_bands(h->P);
            if (!std::isfinite(o.split_far_ratio) || (o.split_far_ratio > 0 && o.split_far_ratio < 1)) {
                delete h;
                return fail(NDSI_ERR_INVALID, "ndsi_analyze_batched: split_far_ratio must be 0, negative or >= 1");
            }
            if (o.split_far_ratio == 0) o.split_far_ratio = kSplitFarRatio;
            h->P.opt.split_slices = o.split_slices;
            h->P.opt.split_bands = o.split_bands;
            h->P.opt.split_far_ratio = o.split_far_ratio;
            setup_split(h, o);
        }
        *plan_out = h;
    } catch (const std::bad_alloc&) {
        return fail(NDSI_ERR_OOM, "ndsi_analyze_batched: out of host memory");
    }
    return NDSI_OK;
}

static int density_batched_entry(ndsi_plan* h, const double* H, const double* S, const double* mu,
                                 const double* kT, int32_t n_poles, const PoleRange* range, double* rho_out,
                                 double* n_elec_out, void* stream) {
    if (!h || !H || !S || !mu || !kT || !rho_out || n_poles < 1)
        return fail(NDSI_ERR_INVALID, "ndsi_density_batched: invalid argument");
    const int32_t ns = h->P.n_systems;
    for (int32_t i = 0; i < ns; ++i)
        if (!(kT[i] > 0) || !std::isfinite(mu[i])) return fail(NDSI_ERR_INVALID, "ndsi_density_batched: bad mu/kT");
    if (foreign_device_ptr(rho_out) || foreign_device_ptr(n_elec_out))
        return fail(NDSI_ERR_INVALID, "ndsi_density_batched: an output is device memory of another GPU");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int rc = upload_tables(h);
    if (rc) return rc;
    const double *Hd, *Sd;
    rc = device_inputs(h, H, S, &Hd, &Sd, st);
    if (rc) return rc;
    const bool rho_dev = is_device_ptr(rho_out);
    const bool ne_dev = n_elec_out && is_device_ptr(n_elec_out);
    rc = ensure_stage(h, 3 * h->P.nnz + 8 + ns);
    if (rc) return rc;
    double* rho_d = rho_dev ? rho_out : h->stage + 2 * h->P.nnz;
    double* ne_d = ne_dev ? n_elec_out : h->stage + 3 * h->P.nnz;
    std::vector<double> muv(mu, mu + ns), ktv(kT, kT + ns);
    rc = density_impl(h, Hd, Sd, muv.data(), ktv.data(), n_poles, rho_d, ne_d, st, nullptr, range);
    if (rc) return rc;
    if (!rho_dev) NDSI_CK(cudaMemcpyAsync(rho_out, rho_d, sizeof(double) * h->P.nnz, cudaMemcpyDeviceToHost, st));
    if (n_elec_out && !ne_dev) NDSI_CK(cudaMemcpyAsync(n_elec_out, ne_d, sizeof(double) * ns, cudaMemcpyDeviceToHost, st));
    NDSI_CK(cudaStreamSynchronize(st));
    return NDSI_OK;
}

int ndsi_density_batched(ndsi_plan* h, const double* H, const double* S, const double* mu, const double* kT,
                         int32_t n_poles, double* rho_out, double* n_elec_out, void* stream) {
    return density_batched_entry(h, H, S, mu, kT, n_poles, nullptr, rho_out, n_elec_out, stream);
}

int ndsi_density_batched_poles(ndsi_plan* h, const double* H, const double* S, const double* mu,
                               const double* kT, int32_t n_poles, int32_t pole_begin, int32_t pole_end,
                               int32_t with_m0, double* rho_out, double* n_elec_out, void* stream) {
    if (pole_begin < 0 || pole_end > n_poles || pole_begin > pole_end)
        return fail(NDSI_ERR_INVALID, "ndsi_density_batched_poles: bad pole range");
    PoleRange r;
    r.begin = pole_begin;
    r.end = pole_end;
    r.m0 = with_m0 != 0;
    return density_batched_entry(h, H, S, mu, kT, n_poles, &r, rho_out, n_elec_out, stream);
}

int ndsi_plan_info(const ndsi_plan* h, ndsi_plan_summary* out) {
    if (!h || !out) return fail(NDSI_ERR_INVALID, "ndsi_plan_info: NULL argument");
    const Plan& P = h->P;
    out->n = P.n;
    out->nnz = P.nnz;
    out->n_atoms = P.n_atoms;
    out->n_nodes = P.n_nodes;
    out->n_levels = P.n_levels;
    out->max_front = P.max_front;
    out->front_elems = P.front_total;
    out->flops_per_pole = P.flops_per_pole;
    out->bytes_per_pole = P.bytes_per_pole;
    out->n_launches = static_cast<int32_t>(P.launches.size());
    out->n_systems = P.n_systems;
    out->split_slices = P.opt.precision == NDSI_PREC_SPLIT ? P.opt.split_slices : 0;
    out->split_bands = P.opt.precision == NDSI_PREC_SPLIT
                           ? (P.opt.split_bands != 0 ? P.opt.split_bands : P.opt.split_slices)
                           : 0;
    return NDSI_OK;
}

int ndsi_plan_export(const ndsi_plan* h, int32_t what, void* out) {
    if (!h || !out) return fail(NDSI_ERR_INVALID, "ndsi_plan_export: NULL argument");
    const Plan& P = h->P;
    if (P.n_systems != 1 && what != NDSI_EXPORT_SCHEDULE && what != NDSI_EXPORT_LEVEL && what != NDSI_EXPORT_PARENT &&
        what != NDSI_EXPORT_TILE_SHAPES)
        return fail(NDSI_ERR_INVALID, "ndsi_plan_export: ordering tables are per system; not available for a batch");
    switch (what) {
        case NDSI_EXPORT_PERM_ATOMS: std::memcpy(out, P.perm_atoms.data(), bytes_of(P.perm_atoms)); break;
        case NDSI_EXPORT_PERM_BASIS: std::memcpy(out, P.perm_basis.data(), bytes_of(P.perm_basis)); break;
        case NDSI_EXPORT_NODE_ATOMS: std::memcpy(out, P.node_atom_first.data(), bytes_of(P.node_atom_first)); break;
        case NDSI_EXPORT_PARENT: std::memcpy(out, P.parent.data(), bytes_of(P.parent)); break;
        case NDSI_EXPORT_STRUCT_PTR: std::memcpy(out, P.struct_ptr.data(), bytes_of(P.struct_ptr)); break;
        case NDSI_EXPORT_STRUCT_ATOMS:
            if (!P.struct_atoms.empty()) std::memcpy(out, P.struct_atoms.data(), bytes_of(P.struct_atoms));
            break;
        case NDSI_EXPORT_LEVEL: std::memcpy(out, P.level.data(), bytes_of(P.level)); break;
        case NDSI_EXPORT_SCHEDULE: {
            int32_t* o = static_cast<int32_t*>(out);
            for (size_t i = 0; i < P.launches.size(); ++i) {
                o[4 * i + 0] = P.launches[i].kind;
                o[4 * i + 1] = P.launches[i].level;
                o[4 * i + 2] = P.launches[i].tag;
                o[4 * i + 3] = static_cast<int32_t>(P.launches[i].count);
            }
            break;
        }
        case NDSI_EXPORT_TILE_SHAPES: {
            int32_t* o = static_cast<int32_t*>(out);
            const bool split = P.opt.precision == NDSI_PREC_SPLIT;
            for (size_t i = 0; i < P.launches.size(); ++i) {
                const Launch& l = P.launches[i];
                if (l.kind != L_GEMM) {
                    o[i] = -1;
                } else if (!split || !split_eligible(l) || !h->SP.use_split[i]) {
                    o[i] = 0;
                } else {
                    o[i] = h->SP.steps[h->SP.step_of_launch[i]].nc;
                }
            }
            break;
        }
        default: return fail(NDSI_ERR_INVALID, "ndsi_plan_export: unknown item");
    }
    return NDSI_OK;
}

int ndsi_factor_poles(ndsi_plan* h, const double* H, const double* S, const double* z, int32_t n_poles,
                      ndsi_factors** f_out, void* stream) {
    if (!h || !H || !S || !z || !f_out || n_poles < 1)
        return fail(NDSI_ERR_INVALID, "ndsi_factor_poles: invalid argument");
    *f_out = nullptr;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int rc = upload_tables(h);
    if (rc) return rc;
    const int64_t need = int64_t(n_poles) * bytes_per_pole(h);
    if (h->P.opt.max_workspace_bytes > 0 && need > h->P.opt.max_workspace_bytes)
        return fail(NDSI_ERR_OOM, "ndsi_factor_poles: factors exceed max_workspace_bytes");
    std::unique_ptr<ndsi_factors> f(new (std::nothrow) ndsi_factors());
    if (!f) return fail(NDSI_ERR_OOM, "ndsi_factor_poles: out of host memory");
    f->plan = h;
    f->np = n_poles;
    f->split_gen = h->SP.generation;
    rc = alloc_workspace(f->W, h->P, n_poles);
    if (rc) {
        free_workspace(f->W);
        return rc;
    }
    if (cudaMalloc(&f->zd, sizeof(double2) * n_poles) != cudaSuccess) {
        cudaGetLastError();
        free_workspace(f->W);
        return fail(NDSI_ERR_OOM, "ndsi_factor_poles: cudaMalloc of pole array failed");
    }
    auto cleanup = [&]() {
        free_workspace(f->W);
        split_free(f->SB);
        cudaFree(f->zd);
    };
    if (h->P.opt.precision == NDSI_PREC_SPLIT) {
        cudaError_t e = split_alloc(f->SB, h->SP.steps, h->P.opt.split_slices, n_poles);
        if (e != cudaSuccess) {
            cudaGetLastError();
            cleanup();
            return fail(e == cudaErrorMemoryAllocation ? NDSI_ERR_OOM : NDSI_ERR_CUDA,
                        std::string("ndsi_factor_poles: split buffers: ") + cudaGetErrorString(e));
        }
    }
    if (cudaMemcpyAsync(f->zd, z, sizeof(double2) * n_poles, cudaMemcpyHostToDevice, st) != cudaSuccess) {
        cleanup();
        return fail(NDSI_ERR_CUDA, "ndsi_factor_poles: pole upload failed");
    }
    const double *Hd, *Sd;
    rc = device_inputs(h, H, S, &Hd, &Sd, st);
    if (!rc) rc = run_phase(h, f->W, f->SB, 0, Hd, Sd, f->zd, 0, n_poles, st);
    if (rc) {
        cleanup();
        return rc;
    }
    *f_out = f.release();
    return NDSI_OK;
}

int ndsi_selinv(ndsi_factors* f, double* G_out, void* stream) {
    if (!f || !f->plan) return fail(NDSI_ERR_INVALID, "ndsi_selinv: NULL factors");
    ndsi_plan* h = f->plan;
    if (f->split_gen != h->SP.generation)
        return fail(NDSI_ERR_INVALID, "ndsi_selinv: the plan's split schedule was retuned after these factors were made");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int rc = run_phase(h, f->W, f->SB, 1, nullptr, nullptr, f->zd, 0, f->np, st);
    f->inverted = true;
    if (rc) return rc;
    if (G_out) {
        const bool dev = is_device_ptr(G_out);
        double2* dst = reinterpret_cast<double2*>(G_out);
        double2* tmp = nullptr;
        const size_t bytes = sizeof(double2) * static_cast<size_t>(f->np) * h->P.nnz;
        if (!dev) NDSI_CK(cudaMalloc(&tmp, bytes));
        NDSI_CK(launch_gather_pattern(h->P, h->T, f->W, f->np, dev ? dst : tmp, 0, st));
        if (!dev) {
            cudaError_t e = cudaMemcpyAsync(G_out, tmp, bytes, cudaMemcpyDeviceToHost, st);
            cudaError_t e2 = cudaStreamSynchronize(st);
            cudaFree(tmp);
            NDSI_CK(e);
            NDSI_CK(e2);
        }
    }
    return check_status(h, st);
}

static int density_entry(ndsi_plan* h, const double* H, const double* S, double mu, double kT, int32_t n_poles,
                         const PoleRange* range, double* rho_out, double* n_elec_out, void* stream) {
    if (foreign_device_ptr(rho_out) || foreign_device_ptr(n_elec_out))
        return fail(NDSI_ERR_INVALID, "ndsi_density: an output is device memory of another GPU");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int rc = upload_tables(h);
    if (rc) return rc;
    const double *Hd, *Sd;
    rc = device_inputs(h, H, S, &Hd, &Sd, st);
    if (rc) return rc;
    const bool rho_dev = is_device_ptr(rho_out);
    const bool ne_dev = n_elec_out && is_device_ptr(n_elec_out);
    rc = ensure_stage(h, 3 * h->P.nnz + 8);
    if (rc) return rc;
    double* rho_d = rho_dev ? rho_out : h->stage + 2 * h->P.nnz;
    double* ne_d = ne_dev ? n_elec_out : h->stage + 3 * h->P.nnz;
    if (h->P.n_systems != 1) return fail(NDSI_ERR_INVALID, "ndsi_density: batched plan, use ndsi_density_batched");
    rc = density_impl(h, Hd, Sd, &mu, &kT, n_poles, rho_d, ne_d, st, nullptr, range);
    if (rc) return rc;
    if (!rho_dev) NDSI_CK(cudaMemcpyAsync(rho_out, rho_d, sizeof(double) * h->P.nnz, cudaMemcpyDeviceToHost, st));
    if (n_elec_out && !ne_dev) NDSI_CK(cudaMemcpyAsync(n_elec_out, ne_d, sizeof(double), cudaMemcpyDeviceToHost, st));
    NDSI_CK(cudaStreamSynchronize(st));
    return NDSI_OK;
}

int ndsi_density(ndsi_plan* h, const double* H, const double* S, double mu, double kT, int32_t n_poles,
                 double* rho_out, double* n_elec_out, void* stream) {
    if (!h || !H || !S || !rho_out || n_poles < 1 || !(kT > 0) || !std::isfinite(mu))
        return fail(NDSI_ERR_INVALID, "ndsi_density: invalid argument");
    return density_entry(h, H, S, mu, kT, n_poles, nullptr, rho_out, n_elec_out, stream);
}

int ndsi_density_poles(ndsi_plan* h, const double* H, const double* S, double mu, double kT, int32_t n_poles,
                       int32_t pole_begin, int32_t pole_end, int32_t with_m0, double* rho_out,
                       double* n_elec_out, void* stream) {
    if (!h || !H || !S || !rho_out || n_poles < 1 || !(kT > 0) || !std::isfinite(mu) || pole_begin < 0 ||
        pole_end > n_poles || pole_begin > pole_end)
        return fail(NDSI_ERR_INVALID, "ndsi_density_poles: invalid argument");
    PoleRange r;
    r.begin = pole_begin;
    r.end = pole_end;
    r.m0 = with_m0 != 0;
    return density_entry(h, H, S, mu, kT, n_poles, &r, rho_out, n_elec_out, stream);
}

int ndsi_pole_shard(int32_t n_poles, int32_t rank, int32_t world, int32_t* pole_begin, int32_t* pole_end,
                    int32_t* with_m0) {
    if (n_poles < 1 || world < 1 || rank < 0 || rank >= world || !pole_begin || !pole_end || !with_m0)
        return fail(NDSI_ERR_INVALID, "ndsi_pole_shard: invalid argument");
    // contiguous ranges whose sizes differ by at most one: rank r takes [r M / W, (r + 1) M / W);
    // the first rank of the smaller size (the first rank when all are equal) also takes M0
    auto lo = [&](int32_t r) { return static_cast<int32_t>((static_cast<int64_t>(r) * n_poles) / world); };
    int32_t m0_rank = 0, min_cnt = n_poles + 1;
    for (int32_t r = 0; r < world; ++r) {
        const int32_t cnt = lo(r + 1) - lo(r);
        if (cnt < min_cnt) {
            min_cnt = cnt;
            m0_rank = r;
        }
    }
    *pole_begin = lo(rank);
    *pole_end = lo(rank + 1);
    *with_m0 = rank == m0_rank ? 1 : 0;
    return NDSI_OK;
}

int ndsi_density_energy(ndsi_plan* h, const double* H, const double* S, double mu, double kT, int32_t n_poles,
                        double* rho_out, double* e_out, double* n_elec_out, void* stream) {
    if (!h || !H || !S || !rho_out || !e_out || n_poles < 1 || !(kT > 0) || !std::isfinite(mu))
        return fail(NDSI_ERR_INVALID, "ndsi_density_energy: invalid argument");
    if (h->P.n_systems != 1) return fail(NDSI_ERR_INVALID, "ndsi_density_energy: batched plan");
    if (foreign_device_ptr(rho_out) || foreign_device_ptr(e_out) || foreign_device_ptr(n_elec_out))
        return fail(NDSI_ERR_INVALID, "ndsi_density_energy: an output is device memory of another GPU");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int rc = upload_tables(h);
    if (rc) return rc;
    const double *Hd, *Sd;
    rc = device_inputs(h, H, S, &Hd, &Sd, st);
    if (rc) return rc;
    const int64_t nnz = h->P.nnz;
    const bool rho_dev = is_device_ptr(rho_out), e_dev = is_device_ptr(e_out);
    const bool ne_dev = n_elec_out && is_device_ptr(n_elec_out);
    rc = ensure_stage(h, 4 * nnz + 8);
    if (rc) return rc;
    double* rho_d = rho_dev ? rho_out : h->stage + 2 * nnz;
    double* ne_d = ne_dev ? n_elec_out : h->stage + 3 * nnz;
    double* e_d = e_dev ? e_out : h->stage + 3 * nnz + 8;
    rc = density_impl(h, Hd, Sd, &mu, &kT, n_poles, rho_d, ne_d, st, e_d);
    if (rc) return rc;
    if (!rho_dev) NDSI_CK(cudaMemcpyAsync(rho_out, rho_d, sizeof(double) * nnz, cudaMemcpyDeviceToHost, st));
    if (!e_dev) NDSI_CK(cudaMemcpyAsync(e_out, e_d, sizeof(double) * nnz, cudaMemcpyDeviceToHost, st));
    if (n_elec_out && !ne_dev) NDSI_CK(cudaMemcpyAsync(n_elec_out, ne_d, sizeof(double), cudaMemcpyDeviceToHost, st));
    NDSI_CK(cudaStreamSynchronize(st));
    return NDSI_OK;
}

}  // extern "C"

namespace ndsi {
// rho(mu) and Tr(rho S) of every system of the plan (mu[s], kT[s]) for device inputs and
// outputs (ne_d[s] per system); synchronises the stream.
int density_impl(ndsi_plan* h, const double* Hd, const double* Sd, const double* mu, const double* kT,
                 int32_t n_poles, double* rho_d, double* ne_d, cudaStream_t st, double* e_d,
                 const PoleRange* range) {
    int rc;
    const int32_t ns = h->P.n_systems;
    if (e_d && ns != 1) return fail(NDSI_ERR_INVALID, "energy density: single-system plans only");
    const int32_t pb = range ? range->begin : 0;
    const int32_t pe = range ? range->end : n_poles;
    const bool with_m0 = range ? range->m0 : true;
    if (range && (e_d || pb < 0 || pe > n_poles || pb > pe))
        return fail(NDSI_ERR_INVALID, "density: bad pole range");
    if (pe - pb + (with_m0 ? 1 : 0) == 0) {
        // an empty share of the sum: rho = 0, Tr(rho S) = 0 for every system
        NDSI_CK(cudaMemsetAsync(rho_d, 0, sizeof(double) * h->P.nnz, st));
        NDSI_CK(cudaMemsetAsync(ne_d, 0, sizeof(double) * ns, st));
        return check_status(h, st);
    }
    // Energy density matrix (Eq. 10): the same points with weights -4 R_p alpha_p kT, kappa on the
    // M0 point, and the first moment M1 from three more points z = Re, -Re, i Re with
    // M1 = (Re^2 / 4) [G(Re) + G(-Re) - 2 Re G(i Re)] (the four points Re i^k annihilate every
    // moment except M1, M5, ...: truncation ~ (spectral radius / Re)^4 |M1|).  Re is 1000 x the
    // Gershgorin bound of the pencil's spectrum, computed on the device.
    double Re = 0.0;
    if (e_d) {
        if (!h->gersh) NDSI_CK(cudaMalloc(&h->gersh, 2 * sizeof(unsigned long long)));
        NDSI_CK(cudaMemsetAsync(h->gersh, 0, 2 * sizeof(unsigned long long), st));
        NDSI_CK(launch_gershgorin(h->T, h->P.n, Hd, Sd, h->gersh, st));
        unsigned long long keys[2];
        NDSI_CK(cudaMemcpyAsync(keys, h->gersh, sizeof(keys), cudaMemcpyDeviceToHost, st));
        NDSI_CK(cudaStreamSynchronize(st));
        const double hmax = gershgorin_value(keys[0]), smin = -gershgorin_value(keys[1]);
        const double radius = hmax / (smin > 1e-3 ? smin : 1e-3);
        Re = 1000.0 * std::max(radius, 1e-3);
    }
    // poles of Eq. 7 (cached per M) -> points alpha_p and weights w_p of Eq. 8, plus iR for M0
    if (h->pole_M != n_poles) {
        h->pole_z.assign(n_poles, 0.0);
        h->pole_R.assign(n_poles, 0.0);
        std::string err;
        rc = cf_poles(n_poles, h->pole_z.data(), h->pole_R.data(), err);
        if (rc) return fail(rc, err);
        h->pole_M = n_poles;
    }
    // Points of this call, in two groups: first those that need every slice of a split plan
    // (poles pb..pf-1 near the real axis, M0, the three moment points), then the far poles pf..pe-1,
    // which a split plan runs with one slice fewer (ndsi_options.split_far_ratio; pf = pe when the
    // plan is FP64, the option is off or no slice can be dropped).
    int32_t pf = pe;
    if (h->P.opt.precision == NDSI_PREC_SPLIT && h->P.opt.split_far_ratio > 0 && h->P.opt.split_slices > 4) {
        pf = pb;
        while (pf < pe && h->pole_z[pf] < h->P.opt.split_far_ratio * h->pole_z[0]) ++pf;
    }
    const int32_t n_near = (pf - pb) + (with_m0 ? 1 : 0) + (e_d ? 3 : 0);
    const int32_t nq = n_near + (pe - pf);
    std::vector<double2> zq(static_cast<size_t>(ns) * nq), cq(static_cast<size_t>(ns) * nq),
        ceq(static_cast<size_t>(ns) * nq, make_double2(0.0, 0.0));
    const double R = h->P.opt.m0_radius;
    for (int32_t sy = 0; sy < ns; ++sy) {
        double2* z = zq.data() + static_cast<size_t>(sy) * nq;
        double2* c = cq.data() + static_cast<size_t>(sy) * nq;
        double2* ce = ceq.data() + static_cast<size_t>(sy) * nq;
        double kappa = 0.0;
        for (int32_t p = 0; p < n_poles; ++p) kappa += 4.0 * kT[sy] * h->pole_R[p];
        auto put_pole = [&](int32_t q, int32_t p) {
            z[q] = make_double2(mu[sy], h->pole_z[p] * kT[sy]);
            c[q] = make_double2(-4.0 * h->pole_R[p] * kT[sy], 0.0);
            // -4 R_p kT alpha_p: Re(ce G) = -4 R_p kT Re(alpha_p G)
            ce[q] = make_double2(-4.0 * h->pole_R[p] * kT[sy] * mu[sy], -4.0 * h->pole_R[p] * kT[sy] * z[q].y);
        };
        int32_t q = 0;
        for (int32_t p = pb; p < pf; ++p) put_pole(q++, p);
        if (with_m0) {
            z[q] = make_double2(0.0, R);
            c[q] = make_double2(0.0, R);
            ce[q] = make_double2(0.0, kappa * R);  // kappa M0, M0 = Re(i R G(i R))
            ++q;
        }
        if (e_d) {
            z[q] = make_double2(Re, 0.0);
            z[q + 1] = make_double2(-Re, 0.0);
            z[q + 2] = make_double2(0.0, Re);
            c[q] = c[q + 1] = c[q + 2] = make_double2(0.0, 0.0);
            ce[q] = ce[q + 1] = make_double2(0.25 * Re * Re, 0.0);
            ce[q + 2] = make_double2(-0.5 * Re * Re, 0.0);
            q += 3;
        }
        for (int32_t p = pf; p < pe; ++p) put_pole(q++, p);
    }
    // chunk the points to the workspace cap
    const int64_t per_pole = bytes_per_pole(h);
    int64_t cap = workspace_cap(h);
    int32_t chunk = static_cast<int32_t>(std::min<int64_t>(nq, std::max<int64_t>(1, cap / per_pole)));
    if (cap < per_pole) return fail(NDSI_ERR_OOM, "ndsi_density: one pole does not fit the workspace cap");
    rc = alloc_workspace(h->W, h->P, chunk);
    if (rc) return rc;
    if (h->P.opt.precision == NDSI_PREC_SPLIT) NDSI_CK(split_alloc(h->SB, h->SP.steps, h->P.opt.split_slices, chunk));
    if (h->cw_cap < ns * nq) {
        if (h->cw) cudaFree(h->cw);
        if (h->zw) cudaFree(h->zw);
        if (h->cew) cudaFree(h->cew);
        h->cw = h->zw = h->cew = nullptr;
        h->cw_cap = 0;
        NDSI_CK(cudaMalloc(&h->cw, sizeof(double2) * ns * nq));
        NDSI_CK(cudaMalloc(&h->zw, sizeof(double2) * ns * nq));
        NDSI_CK(cudaMalloc(&h->cew, sizeof(double2) * ns * nq));
        h->cw_cap = ns * nq;
    }
    // per-system partial-trace ranges of the reduction scratch
    std::vector<int> part_off(ns + 1, 0);
    for (int32_t sy = 0; sy < ns; ++sy)
        part_off[sy + 1] = part_off[sy] + accumulate_blocks(h->P.sys_nnz_first[sy + 1] - h->P.sys_nnz_first[sy]);
    if (!h->partials) NDSI_CK(cudaMalloc(&h->partials, sizeof(double) * (part_off[ns] + 1)));
    // the point tables go through pinned staging, so the copies are asynchronous and the host
    // can run a sweep ahead of the GPU; the staging is rewritten only after the previous call's
    // copies have executed
    {
        const size_t cnt = static_cast<size_t>(ns) * nq;
        if (h->pin_cap < cnt) {
            if (h->pin) cudaFreeHost(h->pin);
            h->pin = nullptr;
            h->pin_cap = 0;
            NDSI_CK(cudaMallocHost(&h->pin, sizeof(double2) * 3 * cnt));
            h->pin_cap = cnt;
        }
        if (!h->pin_ev) NDSI_CK(cudaEventCreateWithFlags(&h->pin_ev, cudaEventDisableTiming));
        NDSI_CK(cudaEventSynchronize(h->pin_ev));
        std::memcpy(h->pin, zq.data(), sizeof(double2) * cnt);
        std::memcpy(h->pin + cnt, cq.data(), sizeof(double2) * cnt);
        if (e_d) std::memcpy(h->pin + 2 * cnt, ceq.data(), sizeof(double2) * cnt);
        NDSI_CK(cudaMemcpyAsync(h->zw, h->pin, sizeof(double2) * cnt, cudaMemcpyHostToDevice, st));
        NDSI_CK(cudaMemcpyAsync(h->cw, h->pin + cnt, sizeof(double2) * cnt, cudaMemcpyHostToDevice, st));
        if (e_d) NDSI_CK(cudaMemcpyAsync(h->cew, h->pin + 2 * cnt, sizeof(double2) * cnt, cudaMemcpyHostToDevice, st));
        NDSI_CK(cudaEventRecord(h->pin_ev, st));
    }
    if (h->graphs && !h->prof.on) {
        // replay the captured sweep; points and weights are read from zw / cw at run time
        const std::vector<const void*> key = {Hd, Sd, rho_d, ne_d, e_d, h->W.fronts, h->W.scr, h->SB.sliceA,
                                              h->SB.sliceB, h->cw, h->zw, h->cew, h->partials,
                                              reinterpret_cast<const void*>(static_cast<intptr_t>(nq)),
                                              reinterpret_cast<const void*>(static_cast<intptr_t>(chunk)),
                                              reinterpret_cast<const void*>(static_cast<intptr_t>(n_near))};
        if (!h->graph || h->graph_key != key) {
            if (h->graph) cudaGraphExecDestroy(h->graph);
            h->graph = nullptr;
            if (!h->cap_stream) NDSI_CK(cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
            NDSI_CK(cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
            rc = sweep(h, Hd, Sd, nq, n_near, chunk, part_off, rho_d, ne_d, e_d, h->cap_stream);
            cudaGraph_t g = nullptr;
            const cudaError_t ec = cudaStreamEndCapture(h->cap_stream, &g);
            if (rc || ec != cudaSuccess) {
                if (g) cudaGraphDestroy(g);
                if (rc) return rc;
                NDSI_CK(ec);
            }
            size_t nodes = 0;
            cudaGraphGetNodes(g, nullptr, &nodes);
            const cudaError_t ei = cudaGraphInstantiate(&h->graph, g, 0);
            cudaGraphDestroy(g);
            NDSI_CK(ei);
            h->graph_key = key;
            h->graph_nodes = static_cast<int64_t>(nodes);
        }
        NDSI_CK(cudaGraphLaunch(h->graph, st));
        return check_status(h, st);
    }
    rc = sweep(h, Hd, Sd, nq, n_near, chunk, part_off, rho_d, ne_d, e_d, st);
    if (rc) return rc;
    return check_status(h, st);
}

// One density sweep over all points, chunked: factor, selected inversion and residue sum per
// chunk, then the per-system electron counts.  Points [0, n_near) run with the plan's slice
// count, the far poles [n_near, nq) of a split plan with one slice fewer; no chunk spans both.
// Only stream-ordered work: it is also the body of the captured graph.
int sweep(ndsi_plan* h, const double* Hd, const double* Sd, int32_t nq, int32_t n_near, int32_t chunk,
          const std::vector<int>& part_off, double* rho_d, double* ne_d, double* e_d, cudaStream_t st) {
    int rc;
    const int32_t ns = h->P.n_systems;
    for (int32_t q0 = 0; q0 < nq;) {
        const bool far = q0 >= n_near;
        const int32_t np = std::min(chunk, (far ? nq : n_near) - q0);
        const int slices = far ? h->P.opt.split_slices - 1 : 0;
        rc = run_phase(h, h->W, h->SB, 0, Hd, Sd, h->zw + q0, nq, np, st, slices);
        if (!rc) rc = run_phase(h, h->W, h->SB, 1, Hd, Sd, h->zw + q0, nq, np, st, slices);
        if (rc) return rc;
        const int last = q0 + np >= nq;
        for (int32_t sy = 0; sy < ns; ++sy) {
            const int64_t k0 = h->P.sys_nnz_first[sy], cnt = h->P.sys_nnz_first[sy + 1] - k0;
            const double acc_bytes = static_cast<double>(cnt) * (8.0 + 16.0 * np + 8.0 + 8.0 + (q0 > 0 ? 8.0 : 0.0));
            NDSI_CK(timed(h->prof, "accumulate", 2.0 * np * cnt, acc_bytes, st, [&]() {
                return launch_accumulate(h->P, h->T, h->W, np, h->cw + static_cast<size_t>(sy) * nq + q0, Sd, rho_d,
                                         q0 > 0 ? 1 : 0, last, h->partials + part_off[sy], st, k0, cnt);
            }));
            if (e_d)
                NDSI_CK(timed(h->prof, "accumulate", 2.0 * np * cnt, acc_bytes, st, [&]() {
                    return launch_accumulate(h->P, h->T, h->W, np, h->cew + static_cast<size_t>(sy) * nq + q0, Sd,
                                             e_d, q0 > 0 ? 1 : 0, 0, nullptr, st, k0, cnt);
                }));
        }
        q0 += np;
    }
    for (int32_t sy = 0; sy < ns; ++sy) {
        const int nblk = part_off[sy + 1] - part_off[sy];
        NDSI_CK(timed(h->prof, "reduce", static_cast<double>(nblk), 8.0 * nblk, st,
                      [&]() { return launch_reduce(h->partials + part_off[sy], nblk, ne_d + sy, st); }));
    }
    return NDSI_OK;
}
}  // namespace ndsi

extern "C" {

int ndsi_mu_features(ndsi_plan* h, const double* H, const double* S, double n_electrons, double kT,
                     int32_t n_vectors, uint64_t seed, float* feat_out, void* stream) {
    if (!h || !H || !S || !feat_out || n_vectors < 1 || !(kT > 0) || h->P.n_systems != 1)
        return fail(NDSI_ERR_INVALID, "ndsi_mu_features: invalid argument");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int rc = upload_tables(h);
    if (rc) return rc;
    const double *Hd, *Sd;
    rc = device_inputs(h, H, S, &Hd, &Sd, st);
    if (rc) return rc;
    const bool dev = is_device_ptr(feat_out);
    float* fd = feat_out;
    if (!dev) NDSI_CK(cudaMalloc(&fd, sizeof(float) * NDSI_MLP_INPUTS));
    rc = mlp_features(h->P, Hd, Sd, h->T.rowptr, h->T.col, n_electrons, kT, n_vectors, seed, fd, st);
    if (!dev) {
        if (!rc) {
            cudaError_t e = cudaMemcpy(feat_out, fd, sizeof(float) * NDSI_MLP_INPUTS, cudaMemcpyDeviceToHost);
            if (e != cudaSuccess) rc = fail(NDSI_ERR_CUDA, "ndsi_mu_features: readback failed");
        }
        cudaFree(fd);
    }
    return rc;
}

int ndsi_profile_enable(ndsi_plan* h, int32_t enable) {
    if (!h) return fail(NDSI_ERR_INVALID, "ndsi_profile_enable: NULL plan");
    Profiler& pf = h->prof;
    pf.on = enable != 0;
    pf.by_level = enable == 2;
    if (pf.on) {
        pf.names.clear();
        pf.stats.clear();
        pf.pending.clear();
        pf.used = 0;
    }
    return NDSI_OK;
}

int ndsi_profile_read(const ndsi_plan* h, ndsi_profile_entry* out, int32_t max_entries, int32_t* n_out) {
    if (!h || !out || !n_out || max_entries < 0)
        return fail(NDSI_ERR_INVALID, "ndsi_profile_read: invalid argument");
    const Profiler& pf = h->prof;
    int32_t n = 0;
    for (size_t f = 0; f < pf.names.size() && n < max_entries; ++f) {
        const ProfStat& st = pf.stats[f];
        if (st.launches == 0) continue;
        ndsi_profile_entry& e = out[n++];
        std::memset(&e, 0, sizeof(e));
        std::strncpy(e.name, pf.names[f].c_str(), sizeof(e.name) - 1);
        e.launches = st.launches;
        e.ms = st.ms;
        e.flops = st.flops;
        e.bytes = st.bytes;
        e.tensor_flops = st.tensor_flops;
    }
    *n_out = n;
    return NDSI_OK;
}

void ndsi_factors_destroy(ndsi_factors* f) {
    if (!f) return;
    free_workspace(f->W);
    split_free(f->SB);
    if (f->zd) cudaFree(f->zd);
    if (f->solve_buf) cudaFree(f->solve_buf);
    delete f;
}

void ndsi_plan_destroy(ndsi_plan* h) {
    if (!h) return;
    free_workspace(h->W);
    split_free(h->SB);
    if (h->SP.blob) cudaFree(h->SP.blob);
    for (cudaEvent_t e : h->prof.pool) cudaEventDestroy(e);
    if (h->T.blob) cudaFree(h->T.blob);
    if (h->cw) cudaFree(h->cw);
    if (h->zw) cudaFree(h->zw);
    if (h->cew) cudaFree(h->cew);
    if (h->gersh) cudaFree(h->gersh);
    if (h->partials) cudaFree(h->partials);
    if (h->dos_part) cudaFree(h->dos_part);
    if (h->dos_tr) cudaFree(h->dos_tr);
    if (h->dos_z) cudaFree(h->dos_z);
    if (h->point_z) cudaFree(h->point_z);
    if (h->pin) cudaFreeHost(h->pin);
    if (h->pin_ev) cudaEventDestroy(h->pin_ev);
    solve_tables_free(h->ST);
    if (h->stage) cudaFree(h->stage);
    if (h->graph) cudaGraphExecDestroy(h->graph);
    if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
    delete h;
}

int ndsi_autotune(ndsi_plan* h, const double* H, const double* S, double mu, double kT, int32_t n_poles,
                  int32_t* n_split_out, int32_t* n_fp64_out, void* stream) {
    if (!h || !H || !S || n_poles < 1 || !(kT > 0) || !std::isfinite(mu) || h->P.n_systems != 1)
        return fail(NDSI_ERR_INVALID, "ndsi_autotune: invalid argument");
    const size_t nl = h->P.launches.size();
    auto report = [&]() {
        int32_t ns = 0, nf = 0;
        for (size_t li = 0; li < nl; ++li) {
            if (!split_eligible(h->P.launches[li])) continue;
            if (h->P.opt.precision == NDSI_PREC_SPLIT && h->SP.use_split[li]) ++ns;
            else ++nf;
        }
        if (n_split_out) *n_split_out = ns;
        if (n_fp64_out) *n_fp64_out = nf;
    };
    if (h->P.opt.precision != NDSI_PREC_SPLIT) {
        report();
        return NDSI_OK;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int rc = upload_tables(h);
    if (rc) return rc;
    const double *Hd, *Sd;
    rc = device_inputs(h, H, S, &Hd, &Sd, st);
    if (rc) return rc;
    rc = ensure_stage(h, 3 * h->P.nnz + 8);
    if (rc) return rc;
    double* rho_d = h->stage + 2 * h->P.nnz;
    double* ne_d = h->stage + 3 * h->P.nnz;
    // Per-launch event timing of one sweep with every eligible GEMM on the tensor cores and one
    // with every eligible GEMM on the FP64 CUDA cores (each after an untimed warm-up sweep); each
    // launch then keeps the faster of the two.  Both choices meet the split tolerance, so the
    // result only changes speed.  The profiler's own counters are left as they were.
    // A step whose tensor-core time is already below the least time the FP64 path could take
    // (its issued FP64 flops, 3 of every 4 counted, at the measured DFMA rate) is decided without
    // running it on the FP64 cores: only the other steps are timed there, so the FP64 passes cost
    // about as much as tensor-core ones on large systems.
    double peak = 0.0;
    rc = fp64_rate(st, &peak);
    if (rc) return rc;
    Profiler saved = h->prof;
    h->prof.pending.clear();
    h->prof.used = 0;
    h->prof.on = true;
    std::vector<double> t_split(nl, 0.0), t_fp64(nl, 0.0);
    std::vector<char> decided(nl, 0);
    for (int pass = 0; pass < 2 && !rc; ++pass) {
        std::fill(h->SP.use_split.begin(), h->SP.use_split.end(), 1);
        h->prof.per_launch = pass == 0 ? nullptr : &t_split;
        rc = density_impl(h, Hd, Sd, &mu, &kT, n_poles, rho_d, ne_d, st);
    }
    const double points = static_cast<double>(n_poles) + 1.0;
    for (size_t li = 0; li < nl && !rc; ++li) {
        const Launch& l = h->P.launches[li];
        if (!split_eligible(l)) continue;
        const double fp64_min_ms = 0.75 * l.flops * points / (peak * 1e12) * 1e3;
        decided[li] = t_split[li] <= fp64_min_ms ? 1 : 0;
    }
    for (int pass = 0; pass < 2 && !rc; ++pass) {
        for (size_t li = 0; li < nl; ++li) h->SP.use_split[li] = decided[li];
        h->prof.per_launch = pass == 0 ? nullptr : &t_fp64;
        rc = density_impl(h, Hd, Sd, &mu, &kT, n_poles, rho_d, ne_d, st);
    }
    h->prof.per_launch = nullptr;
    for (size_t li = 0; li < nl; ++li)
        h->SP.use_split[li] = !rc && split_eligible(h->P.launches[li])
                                  ? (decided[li] || t_split[li] <= t_fp64[li] ? 1 : 0)
                                  : 1;
    // Tile shape of each tensor-core step: one accumulator per scale (40 complex columns per
    // tile, the plan default) or five accumulator bands (48 columns, a floor near 2^-43 of the
    // result, well inside the split tolerance).  The wider tile carries more multiply-adds per
    // operand byte; which one is faster depends on the step's shapes, so each step keeps the
    // faster of the two timings.  Plans built with a fixed band count keep it.
    bool per_scale = true;
    for (size_t li = 0; li < nl; ++li)
        if (split_eligible(h->P.launches[li]) && h->SP.bands[li] != 0) per_scale = false;
    if (!rc && per_scale) {
        std::vector<double> t_b5(nl, 0.0);
        for (size_t li = 0; li < nl; ++li)
            if (split_eligible(h->P.launches[li]) && h->SP.use_split[li]) h->SP.bands[li] = 5;
        rc = rebuild_split(h);
        for (int pass = 0; pass < 2 && !rc; ++pass) {
            h->prof.per_launch = pass == 0 ? nullptr : &t_b5;
            rc = density_impl(h, Hd, Sd, &mu, &kT, n_poles, rho_d, ne_d, st);
        }
        h->prof.per_launch = nullptr;
        for (size_t li = 0; li < nl; ++li)
            h->SP.bands[li] = (!rc && h->SP.bands[li] == 5 && t_b5[li] < t_split[li]) ? 5 : 0;
        const int rc2 = rebuild_split(h);
        if (!rc) rc = rc2;
    }
    saved.pool = h->prof.pool;  // events created meanwhile stay owned by the plan
    h->prof = saved;
    h->prof.pending.clear();
    h->prof.used = 0;
    if (h->graph) {
        cudaGraphExecDestroy(h->graph);
        h->graph = nullptr;
        h->graph_key.clear();
        h->graph_nodes = 0;
    }
    if (rc) return rc;
    report();
    return NDSI_OK;
}

int ndsi_graph_enable(ndsi_plan* h, int32_t enable) {
    if (!h) return fail(NDSI_ERR_INVALID, "ndsi_graph_enable: NULL plan");
    h->graphs = enable != 0;
    if (!h->graphs && h->graph) {
        cudaGraphExecDestroy(h->graph);
        h->graph = nullptr;
        h->graph_key.clear();
        h->graph_nodes = 0;
    }
    return NDSI_OK;
}

int ndsi_graph_info(const ndsi_plan* h, int64_t* nodes_out) {
    if (!h || !nodes_out) return fail(NDSI_ERR_INVALID, "ndsi_graph_info: NULL argument");
    *nodes_out = h->graph ? h->graph_nodes : 0;
    return NDSI_OK;
}

int ndsi_plan_check(const ndsi_plan* h) {
    if (!h) return fail(NDSI_ERR_INVALID, "ndsi_plan_check: NULL plan");
    std::string err;
    const int rc = check_plan(h->P, err);
    return rc ? fail(rc, err) : NDSI_OK;
}

const char* ndsi_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"
