// C ABI of libepic.so: argument checking, plan lifetime, device uploads,
// dispatch to the path kernels, host-buffer convenience call, kernel timing.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <new>
#include <string>

#include "epic_internal.h"

namespace {
std::mutex g_err_mu;
std::string g_create_error;  // detail of the last failed epic_plan_create

void set_create_error(const std::string& s)
{
    std::lock_guard<std::mutex> lk(g_err_mu);
    g_create_error = s;
}

template <class T>
cudaError_t upload(T** dst, const T* src, size_t n, size_t* bytes)
{
    *dst = nullptr;
    if (n == 0) return cudaSuccess;
    cudaError_t e = cudaMalloc((void**)dst, n * sizeof(T));
    if (e != cudaSuccess) return e;
    *bytes += n * sizeof(T);
    return cudaMemcpy(*dst, src, n * sizeof(T), cudaMemcpyHostToDevice);
}

void free_path_state(epic_plan_s* p);

void free_plan(epic_plan_s* p)
{
    if (!p) return;
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(p->device);
    cudaDeviceSynchronize();
    cudaFree(p->dt.box);
    cudaFree(p->dt.cell_off);
    cudaFree(p->dt.cell_ptr);
    cudaFree(p->dt.contrib_e);
    cudaFree(p->dt.contrib_w);
    cudaFree(p->dt.twiddle);
    cudaFree(p->dt.first_xy);
    cudaFree(p->dt.w_taps);
    cudaFree(p->dt.jones);
    cudaFree(p->dt.dft_f16);
    free_path_state(p);
    cudaFree(p->tc.status);
    cudaFree(p->stage_volt);
    cudaFree(p->stage_out);
    for (auto& ev : p->events) {
        cudaEventDestroy(ev.start);
        cudaEventDestroy(ev.stop);
    }
    if (p->cap_stream) cudaStreamDestroy(p->cap_stream);
    for (cudaEvent_t ev : p->copy_ev) cudaEventDestroy(ev);
    if (p->copy_stream) cudaStreamDestroy(p->copy_stream);
    cudaSetDevice(cur);
    delete p;
}

// Everything a path owns: the tensor path's tables, the scratch, the recorded graph.
void free_path_state(epic_plan_s* p)
{
    cudaFree(p->tc.a1);
    cudaFree(p->tc.a2);
    cudaFree(p->tc.a1_off);
    cudaFree(p->tc.a2_off);
    cudaFree(p->tc.a2w);
    cudaFree(p->tc.a2w_off);
    cudaFree(p->tc.a1p);
    cudaFree(p->tc.a1p_off);
    cudaFree(p->tc.gtask);
    cudaFree(p->tc.partial);
    cudaFree(p->tc.counters);
    cudaFree(p->tc.gtask_off);
    cudaFree(p->tc.gell_e);
    cudaFree(p->tc.gell_w);
    cudaFree(p->tc.gell_off);
    cudaFree(p->tc.tbox);
    cudaFree(p->tc.wcum);
    cudaFree(p->tc.item_order);
    cudaFree(p->tc.pl_ptr);
    cudaFree(p->tc.pl_off);
    cudaFree(p->tc.pl_e);
    cudaFree(p->tc.pl_w);
    cudaFree(p->scratch);
    int* status = p->tc.status;
    p->tc = epic::TcState{};
    p->tc.status = status;
    p->scratch = nullptr;
    p->scratch_bytes = 0;
    p->chunk_budget = 0;
    p->time_chunk = 0;
    p->slab = 0;
    p->fused_variant = 0;
    p->dt.dft_bytes = 0;
    p->tc_flops_per_sample = 0.0;
    if (p->gexec) cudaGraphExecDestroy(p->gexec);
    p->gexec = nullptr;
    p->g_T = -1;
}

bool is_pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }

epic_status path_setup(epic_plan_s* p)
{
    switch (p->path) {
        case EPIC_PATH_PLAIN_FP32: return epic::plain_setup(p);
        case EPIC_PATH_FUSED_FP32: return epic::fused_setup(p);
        case EPIC_PATH_DFTGEMM_FP16: return epic::dftgemm_setup(p);
    }
    return EPIC_ERR_INVALID_ARG;
}
}  // namespace

namespace epic {
epic_status set_path(epic_plan_s* p, int path)
{
    if (path == p->path) return EPIC_OK;
    if (path != EPIC_PATH_PLAIN_FP32 && path != EPIC_PATH_FUSED_FP32 && path != EPIC_PATH_DFTGEMM_FP16)
        return EPIC_ERR_UNSUPPORTED;
    const int old = p->path;
    cudaDeviceSynchronize();  // nothing of this plan may still run on the state freed here
    free_path_state(p);
    p->path = path;
    epic_status st = path_setup(p);
    if (st == EPIC_OK) return EPIC_OK;
    const std::string why = p->last_error;
    free_path_state(p);
    p->path = old;
    const epic_status back = path_setup(p);
    p->last_error = why;
    return back == EPIC_OK ? st : back;
}
}  // namespace epic

namespace epic {

epic_status cuda_fail(epic_plan_s* p, cudaError_t e, const char* what)
{
    std::string msg = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
    if (p) p->last_error = msg;
    set_create_error(msg);
    return e == cudaErrorMemoryAllocation ? EPIC_ERR_OOM : EPIC_ERR_CUDA;
}

cudaError_t allow_max_smem(const void* fn, int optin)
{
    cudaFuncAttributes fa{};
    cudaError_t e = cudaFuncGetAttributes(&fa, fn);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes);
}

void ev_begin(epic_plan_s* p, const char* name, cudaStream_t s)
{
    if (!p->timing) return;
    if (p->n_events == p->events.size()) {
        if (p->events.size() >= 8192) return;
        KernelEvent ev{name, nullptr, nullptr};
        cudaEventCreate(&ev.start);
        cudaEventCreate(&ev.stop);
        p->events.push_back(ev);
    }
    p->events[p->n_events].name = name;
    if (p->capturing) cudaEventRecordWithFlags(p->events[p->n_events].start, s, cudaEventRecordExternal);
    else cudaEventRecord(p->events[p->n_events].start, s);
}

void ev_end(epic_plan_s* p, cudaStream_t s)
{
    if (!p->timing || p->n_events >= p->events.size()) return;
    if (p->capturing) cudaEventRecordWithFlags(p->events[p->n_events].stop, s, cudaEventRecordExternal);
    else cudaEventRecord(p->events[p->n_events].stop, s);
    ++p->n_events;
}

}  // namespace epic

extern "C" {

const char* epic_status_str(epic_status s)
{
    switch (s) {
        case EPIC_OK: return "EPIC_OK";
        case EPIC_ERR_INVALID_ARG: return "EPIC_ERR_INVALID_ARG";
        case EPIC_ERR_GRID_OVERFLOW: return "EPIC_ERR_GRID_OVERFLOW";
        case EPIC_ERR_OOM: return "EPIC_ERR_OOM";
        case EPIC_ERR_BUSY: return "EPIC_ERR_BUSY";
        case EPIC_ERR_TIMEOUT: return "EPIC_ERR_TIMEOUT";
        case EPIC_ERR_CUDA: return "EPIC_ERR_CUDA";
        case EPIC_ERR_UNSUPPORTED: return "EPIC_ERR_UNSUPPORTED";
        case EPIC_ERR_NOT_FOUND: return "EPIC_ERR_NOT_FOUND";
    }
    return "EPIC_ERR_UNKNOWN";
}

const char* epic_last_error(epic_plan_t plan)
{
    if (plan) return plan->last_error.c_str();
    static thread_local std::string copy;
    std::lock_guard<std::mutex> lk(g_err_mu);
    copy = g_create_error;
    return copy.c_str();
}

epic_status epic_device_query(int* sm_count, int* smem_optin_bytes, int* cc_major, int* cc_minor)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return epic::cuda_fail(nullptr, e, "cudaGetDevice");
    int v = 0;
    if (sm_count) {
        e = cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return epic::cuda_fail(nullptr, e, "cudaDeviceGetAttribute");
        *sm_count = v;
    }
    if (smem_optin_bytes) {
        e = cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        if (e != cudaSuccess) return epic::cuda_fail(nullptr, e, "cudaDeviceGetAttribute");
        *smem_optin_bytes = v;
    }
    if (cc_major) {
        e = cudaDeviceGetAttribute(&v, cudaDevAttrComputeCapabilityMajor, dev);
        if (e != cudaSuccess) return epic::cuda_fail(nullptr, e, "cudaDeviceGetAttribute");
        *cc_major = v;
    }
    if (cc_minor) {
        e = cudaDeviceGetAttribute(&v, cudaDevAttrComputeCapabilityMinor, dev);
        if (e != cudaSuccess) return epic::cuda_fail(nullptr, e, "cudaDeviceGetAttribute");
        *cc_minor = v;
    }
    return EPIC_OK;
}

epic_status epic_plan_create(const epic_plan_desc* d, epic_plan_t* out)
{
    if (!out) {
        set_create_error("out pointer is NULL");
        return EPIC_ERR_INVALID_ARG;
    }
    *out = nullptr;
    auto bad = [](const char* why) {
        set_create_error(why);
        return EPIC_ERR_INVALID_ARG;
    };
    if (!d) return bad("descriptor is NULL");
    if (d->n_ant < 1 || !d->pos_m) return bad("n_ant must be >= 1 and pos_m non-NULL");
    if (d->n_pol != 1 && d->n_pol != 2) return bad("n_pol must be 1 or 2");
    if (d->n_chan < 1 || !d->freq_hz) return bad("n_chan must be >= 1 and freq_hz non-NULL");
    if ((long long)d->n_chan * d->n_pol > 65535) return bad("n_chan x n_pol must be at most 65535");
    if (!is_pow2(d->grid_n) || d->grid_n < 8 || d->grid_n > 512) return bad("grid_n must be a power of two in 8..512");
    if (d->max_time < 1) return bad("max_time must be >= 1");
    if (d->gcf.K < 1 || d->gcf.K > 8 || d->gcf.K > d->grid_n) return bad("gcf.K must be in 1..8");
    if (d->gcf.kind == EPIC_GCF_GAUSSIAN) {
        if (!(d->gcf.sigma_cells > 0.0) || !std::isfinite(d->gcf.sigma_cells)) return bad("gcf.sigma_cells must be > 0");
        if (d->gcf.freq_scaled && !(d->gcf.f_ref_hz > 0.0)) return bad("gcf.f_ref_hz must be > 0 when freq_scaled");
    } else if (d->gcf.kind == EPIC_GCF_TABLE) {
        if (d->gcf.oversample < 1 || d->gcf.oversample > 1024 || !d->gcf.table)
            return bad("TABLE GCF needs oversample in 1..1024 and a table");
    } else {
        return bad("unknown gcf.kind");
    }
    if (d->path < EPIC_PATH_PLAIN_FP32 || d->path > EPIC_PATH_AUTO) return bad("unknown path");
    if (d->input_bits != 0 && d->input_bits != 4 && d->input_bits != 8) return bad("input_bits must be 4 or 8");
    if (d->sub_int < 0 || d->sub_int > d->max_time) return bad("sub_int must be in 0..max_time");
    if ((long long)d->n_ant * d->n_pol > (1 << 20)) return bad("n_ant * n_pol too large");
    if (d->jones && d->n_pol != 2) return bad("a polarisation-mixing kernel needs n_pol == 2");
    if (d->jones)
        for (size_t i = 0; i < (size_t)d->n_chan * d->n_ant * 8; ++i)
            if (!std::isfinite(d->jones[i])) return bad("jones must be finite");
    for (int c = 0; c < d->n_chan; ++c) {
        if (!(d->freq_hz[c] > 0.0) || !std::isfinite(d->freq_hz[c])) return bad("freq_hz must be > 0 and finite");
        if (d->cell_m && (!(d->cell_m[c] > 0.0) || !std::isfinite(d->cell_m[c]))) return bad("cell_m must be > 0");
    }
    for (int i = 0; i < 2 * d->n_ant; ++i)
        if (!std::isfinite(d->pos_m[i])) return bad("pos_m must be finite");

    epic_plan_s* p = new (std::nothrow) epic_plan_s();
    if (!p) {
        set_create_error("host allocation failed");
        return EPIC_ERR_OOM;
    }
    p->A = d->n_ant;
    p->P = d->n_pol;
    p->C = d->n_chan;
    p->N = d->grid_n;
    p->K = d->gcf.K;
    p->nprod = d->n_pol == 1 ? 1 : 4;
    p->max_time = d->max_time;
    p->bits = d->input_bits == 8 ? 8 : 4;
    p->sub = d->sub_int;
    p->logN = 0;
    while ((1 << p->logN) < p->N) ++p->logN;
    p->pos.assign(d->pos_m, d->pos_m + 2 * (size_t)d->n_ant);
    p->freq.assign(d->freq_hz, d->freq_hz + d->n_chan);
    if (d->cell_m) p->cell.assign(d->cell_m, d->cell_m + d->n_chan);
    p->gcf = d->gcf;
    if (d->gcf.kind == EPIC_GCF_TABLE) {
        const size_t side = (size_t)d->gcf.K * d->gcf.oversample + 1;
        p->table.assign(d->gcf.table, d->gcf.table + 2 * side * side);
    }
    p->gcf.table = nullptr;
    if (d->jones) p->jones.assign(d->jones, d->jones + (size_t)d->n_chan * d->n_ant * 8);

    std::string err;
    epic_status st = epic::build_geometry(p, &err);
    if (st != EPIC_OK) {
        set_create_error(err);
        delete p;
        return st;
    }

    // device: must be a GB300-class (sm_103) part; this library carries sm_103a code only
    int major = 0, minor = 0;
    st = epic_device_query(&p->sm_count, &p->smem_optin, &major, &minor);
    if (st != EPIC_OK) {
        delete p;
        return st;
    }
    cudaGetDevice(&p->device);
    if (!(major == 10 && minor == 3)) {
        char buf[128];
        snprintf(buf, sizeof buf, "device has compute capability %d.%d; this build carries sm_103a code only", major,
                 minor);
        set_create_error(buf);
        delete p;
        return EPIC_ERR_UNSUPPORTED;
    }

    int path = d->path;
    p->auto_path = path == EPIC_PATH_AUTO;
    if (path == EPIC_PATH_AUTO) path = EPIC_PATH_DFTGEMM_FP16;  // the tensor path where it can run
    p->path = path;

    // shared device tables
    std::vector<int> cell_off, cell_ptr, contrib_e;
    std::vector<float2> contrib_w, tw;
    epic::build_csr(p, cell_off, cell_ptr, contrib_e, contrib_w);
    epic::build_twiddles(p->N, tw);
    std::vector<int4> box(p->C);
    for (int c = 0; c < p->C; ++c) box[c] = make_int4(p->box[c].x0, p->box[c].y0, p->box[c].nx, p->box[c].ny);
    std::vector<int> first_xy((size_t)p->C * p->A);
    for (size_t i = 0; i < first_xy.size(); ++i) first_xy[i] = (p->first_y[i] << 16) | p->first_x[i];
    std::vector<float2> w_taps(p->w_re.size());
    for (size_t i = 0; i < w_taps.size(); ++i) w_taps[i] = make_float2((float)p->w_re[i], (float)p->w_im[i]);
    // polarisation mixing rows: entry 2 (c A + e) + a = (conj J^{a0}, conj J^{a1}) of element e, channel c
    std::vector<float4> jrows(p->jones.size() / 4);
    for (size_t i = 0; i < jrows.size(); ++i) {
        const float* j = &p->jones[4 * i];  // J^{a0} re, im, J^{a1} re, im
        jrows[i] = make_float4(j[0], -j[1], j[2], -j[3]);
    }

    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess) e = upload(&p->dt.box, box.data(), box.size(), &p->table_bytes);
    if (e == cudaSuccess) e = upload(&p->dt.cell_off, cell_off.data(), cell_off.size(), &p->table_bytes);
    if (e == cudaSuccess) e = upload(&p->dt.cell_ptr, cell_ptr.data(), cell_ptr.size(), &p->table_bytes);
    if (e == cudaSuccess) e = upload(&p->dt.contrib_e, contrib_e.data(), contrib_e.size(), &p->table_bytes);
    if (e == cudaSuccess) e = upload(&p->dt.contrib_w, contrib_w.data(), contrib_w.size(), &p->table_bytes);
    if (e == cudaSuccess) e = upload(&p->dt.twiddle, tw.data(), tw.size(), &p->table_bytes);
    if (e == cudaSuccess) e = upload(&p->dt.first_xy, first_xy.data(), first_xy.size(), &p->table_bytes);
    if (e == cudaSuccess) e = upload(&p->dt.w_taps, w_taps.data(), w_taps.size(), &p->table_bytes);
    if (e == cudaSuccess) e = upload(&p->dt.jones, jrows.data(), jrows.size(), &p->table_bytes);
    if (e != cudaSuccess) {
        st = epic::cuda_fail(p, e, "plan table upload");
        free_plan(p);
        return st;
    }

    st = path_setup(p);
    if (st == EPIC_ERR_UNSUPPORTED && p->auto_path) {  // AUTO: the plain FP32 path takes every plan
        free_path_state(p);
        p->path = EPIC_PATH_PLAIN_FP32;
        st = path_setup(p);
    }
    if (st != EPIC_OK) {
        set_create_error(p->last_error);
        free_plan(p);
        return st;
    }
    if (!p->tc.status) {  // every plan has a bounded-wait flag (the tensor path's kernels set it)
        e = cudaMalloc(&p->tc.status, sizeof(int));
        if (e == cudaSuccess) e = cudaMemset(p->tc.status, 0, sizeof(int));
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        st = epic::cuda_fail(p, e, "plan setup");
        free_plan(p);
        return st;
    }
    *out = p;
    return EPIC_OK;
}

epic_status epic_plan_destroy(epic_plan_t plan)
{
    free_plan(plan);
    return EPIC_OK;
}

epic_status epic_plan_get_info(epic_plan_t p, epic_plan_info* info)
{
    if (!p || !info) return EPIC_ERR_INVALID_ARG;
    info->path = p->path;
    info->n_prod = p->nprod;
    info->box_max_x = p->box_max_x;
    info->box_max_y = p->box_max_y;
    info->time_chunk = p->time_chunk;
    info->scratch_bytes = p->scratch_bytes;
    info->device_bytes = p->table_bytes + p->scratch_bytes + p->dt.dft_bytes + p->stage_bytes;
    int nk = 0;
    const int chunks = p->time_chunk > 0 ? (p->max_time + p->time_chunk - 1) / p->time_chunk : 1;
    if (p->path == EPIC_PATH_PLAIN_FP32) nk = 4 * chunks;
    else if (p->path == EPIC_PATH_DFTGEMM_FP16) nk = 2 * chunks * ((p->C + p->tc.cg - 1) / std::max(1, p->tc.cg));
    else nk = p->scratch ? 2 : 1;
    info->n_kernels = nk;
    info->gemm_flops_per_sample = p->path == EPIC_PATH_DFTGEMM_FP16 ? p->tc_flops_per_sample : 0.0;
    info->input_bits = p->bits;
    info->sub_int = p->sub;
    info->pol_mix = p->jones.empty() ? 0 : 1;
    info->tc_kernel = 0;
    info->row_parts = 0;
    if (p->path == EPIC_PATH_DFTGEMM_FP16) {
        info->tc_kernel = p->tc.ws ? p->tc.ws_variant : p->tc.fast ? 4 : 5;
        for (const int4& r : p->tc.tbox_h) info->row_parts = std::max(info->row_parts, r.y);
    }
    return EPIC_OK;
}

}  // extern "C"

namespace epic {
epic_status image_run(epic_plan_s* p, const uint8_t* volt, int T, cudaStream_t s, float* out, unsigned flags,
                      const GroupHooks* hooks)
{
    const bool acc = (flags & EPIC_ACCUMULATE) != 0;
    p->timing = (flags & EPIC_TIME_KERNELS) != 0;
    p->n_events = 0;
    p->last_stream = s;
    if (T == 0) {
        if (!acc && p->sub == 0) {  // an empty block: zero images (with sub-integrations: no image set)
            cudaError_t e = cudaMemsetAsync(out, 0, sizeof(float) * (size_t)p->C * p->nprod * p->N * p->N, s);
            if (e != cudaSuccess) return epic::cuda_fail(p, e, "cudaMemsetAsync(out)");
        }
        return EPIC_OK;
    }
    switch (p->path) {
        case EPIC_PATH_PLAIN_FP32: return epic::plain_run(p, volt, T, s, out, acc);
        case EPIC_PATH_FUSED_FP32: return epic::fused_run(p, volt, T, s, out, acc);
        case EPIC_PATH_DFTGEMM_FP16: return epic::dftgemm_run(p, volt, T, s, out, acc, hooks);
    }
    return EPIC_ERR_INVALID_ARG;
}

void call_scratch_free(CallScratch& c)
{
    cudaFree(c.scratch);
    cudaFree(c.partial);
    cudaFree(c.counters);
    cudaFree(c.status);
    c = CallScratch{};
}

epic_status call_scratch_fit(epic_plan_s* p, CallScratch& c)
{
    const size_t partial = p->tc.partial ? (size_t)p->sm_count * 2 * 4 * 8192 * sizeof(float) : 0;
    auto grow = [&](void** ptr, size_t* have, size_t need, const char* what) -> epic_status {
        if (need <= *have && (*ptr || need == 0)) return EPIC_OK;
        cudaFree(*ptr);
        *ptr = nullptr;
        *have = 0;
        cudaError_t e = cudaMalloc(ptr, need);
        if (e == cudaSuccess) e = cudaMemset(*ptr, 0, need);
        if (e != cudaSuccess) return cuda_fail(p, e, what);
        *have = need;
        return EPIC_OK;
    };
    size_t counters_bytes = c.n_counters * sizeof(int), status_bytes = c.status ? sizeof(int) : 0;
    epic_status st = grow(&c.scratch, &c.scratch_bytes, p->scratch_bytes, "cudaMalloc(call scratch)");
    if (st == EPIC_OK) st = grow((void**)&c.partial, &c.partial_bytes, partial, "cudaMalloc(call partial sums)");
    if (st == EPIC_OK)
        st = grow((void**)&c.counters, &counters_bytes, p->tc.n_counters * sizeof(int), "cudaMalloc(call counters)");
    c.n_counters = counters_bytes / sizeof(int);
    if (st == EPIC_OK) st = grow((void**)&c.status, &status_bytes, sizeof(int), "cudaMalloc(call status)");
    return st;
}

epic_status image_run_with(epic_plan_s* p, CallScratch& c, const uint8_t* volt, int T, cudaStream_t s, float* out,
                           unsigned flags)
{
    // the kernels take these pointers as launch arguments, so swapping them around the
    // launches is all it takes (calls of one plan come from one host thread)
    std::swap(p->scratch, c.scratch);
    std::swap(p->tc.partial, c.partial);
    std::swap(p->tc.counters, c.counters);
    std::swap(p->tc.status, c.status);
    const epic_status st = image_run(p, volt, T, s, out, flags);
    std::swap(p->scratch, c.scratch);
    std::swap(p->tc.partial, c.partial);
    std::swap(p->tc.counters, c.counters);
    std::swap(p->tc.status, c.status);
    return st;
}
}  // namespace epic

extern "C" {

// Read and clear the plan's bounded-wait flag once the calls that may set it are complete:
// EPIC_ERR_TIMEOUT when a kernel's wait ran out since the flag was last cleared.
static epic_status take_timeout(epic_plan_t p)
{
    if (!p->tc.status) return EPIC_OK;
    int flag = 0;
    cudaError_t e = cudaMemcpy(&flag, p->tc.status, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return epic::cuda_fail(p, e, "bounded-wait flag");
    if (!flag) return EPIC_OK;
    e = cudaMemset(p->tc.status, 0, sizeof(int));
    if (e != cudaSuccess) return epic::cuda_fail(p, e, "bounded-wait flag");
    p->last_error = "a device-side bounded wait ran out; the images of that call are incomplete";
    return EPIC_ERR_TIMEOUT;
}

// Timing events the recorded graph will need (created before recording).
static void reserve_events(epic_plan_t p, int T)
{
    size_t n = 8;
    const int chunks = p->time_chunk > 0 ? (T + p->time_chunk - 1) / p->time_chunk : 1;
    if (p->path == EPIC_PATH_PLAIN_FP32) n = 4ull * chunks;
    else if (p->path == EPIC_PATH_DFTGEMM_FP16) n = 2ull * chunks * ((p->C + p->tc.cg - 1) / std::max(1, p->tc.cg));
    n = std::min<size_t>(n + 2, 8192);
    while (p->events.size() < n) {
        epic::KernelEvent ev{"", nullptr, nullptr};
        if (cudaEventCreate(&ev.start) != cudaSuccess) break;
        if (cudaEventCreate(&ev.stop) != cudaSuccess) {
            cudaEventDestroy(ev.start);
            break;
        }
        p->events.push_back(ev);
    }
}

// EPIC_GRAPH: launch the recorded graph, recording (or re-recording) it first
// when the arguments differ from the ones it was recorded for.
static epic_status image_graph(epic_plan_t p, const uint8_t* volt, int T, cudaStream_t s, float* out, unsigned flags)
{
    const unsigned f = flags & ~EPIC_GRAPH;
    p->timing = (f & EPIC_TIME_KERNELS) != 0;
    if (!(p->gexec && p->g_volt == volt && p->g_out == out && p->g_T == T && p->g_flags == f)) {
        if (!p->cap_stream) {
            cudaError_t e = cudaStreamCreateWithFlags(&p->cap_stream, cudaStreamNonBlocking);
            if (e != cudaSuccess) return epic::cuda_fail(p, e, "cudaStreamCreateWithFlags(graph recording)");
        }
        if (p->timing) reserve_events(p, T);
        cudaError_t e = cudaStreamBeginCapture(p->cap_stream, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return epic::cuda_fail(p, e, "cudaStreamBeginCapture");
        p->capturing = true;
        epic_status st = epic::image_run(p, volt, T, p->cap_stream, out, f);
        p->capturing = false;
        cudaGraph_t g = nullptr;
        e = cudaStreamEndCapture(p->cap_stream, &g);
        if (st != EPIC_OK || e != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            cudaGetLastError();
            return st != EPIC_OK ? st : epic::cuda_fail(p, e, "cudaStreamEndCapture");
        }
        if (p->gexec) {
            cudaGraphExecUpdateResultInfo info{};
            if (cudaGraphExecUpdate(p->gexec, g, &info) != cudaSuccess) {
                cudaGetLastError();
                cudaGraphExecDestroy(p->gexec);
                p->gexec = nullptr;
            }
        }
        if (!p->gexec) e = cudaGraphInstantiate(&p->gexec, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            p->gexec = nullptr;
            p->g_T = -1;
            return epic::cuda_fail(p, e, "cudaGraphInstantiate");
        }
        p->g_volt = volt;
        p->g_out = out;
        p->g_T = T;
        p->g_flags = f;
        p->g_events = p->n_events;
    }
    p->n_events = p->g_events;
    p->last_stream = s;
    cudaError_t e = cudaGraphLaunch(p->gexec, s);
    if (e != cudaSuccess) return epic::cuda_fail(p, e, "cudaGraphLaunch");
    return EPIC_OK;
}

static epic_status image_impl(epic_plan_t p, const uint8_t* volt, int T, cudaStream_t s, float* out, unsigned flags)
{
    if ((flags & EPIC_GRAPH) && T > 0) return image_graph(p, volt, T, s, out, flags);
    return epic::image_run(p, volt, T, s, out, flags & ~EPIC_GRAPH);
}

epic_status epic_image(epic_plan_t p, const uint8_t* volt, int T, void* stream, float* out, unsigned flags)
{
    if (!p) return EPIC_ERR_INVALID_ARG;
    if (T < 0 || T > p->max_time) {
        p->last_error = "T must be in 0..max_time";
        return EPIC_ERR_INVALID_ARG;
    }
    if (!out || (T > 0 && !volt)) {
        p->last_error = "NULL voltage or image pointer";
        return EPIC_ERR_INVALID_ARG;
    }
    if (p->sub > 0 && T % p->sub != 0) {
        p->last_error = "T must be a multiple of the plan's sub_int";
        return EPIC_ERR_INVALID_ARG;
    }
    if (flags & ~(EPIC_ACCUMULATE | EPIC_TIME_KERNELS | EPIC_GRAPH)) {
        p->last_error = "unknown flag bits";
        return EPIC_ERR_INVALID_ARG;
    }
    cudaPointerAttributes at{};
    auto on_device = [&](const void* ptr) {
        return cudaPointerGetAttributes(&at, ptr) == cudaSuccess &&
               (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged);
    };
    if (!on_device(out) || (T > 0 && !on_device(volt))) {
        cudaGetLastError();
        p->last_error = "voltage and image pointers must be device memory";
        return EPIC_ERR_INVALID_ARG;
    }
    return image_impl(p, volt, T, (cudaStream_t)stream, out, flags);
}

// epic_image_host for a tensor-path plan of several channel groups: group g's voltages (its
// channel range of every sample, one 2-D copy) go to the device on the plan's copy stream,
// its kernels wait only for them, and its images come back on the copy stream while the next
// group computes; the call's stream waits for the copy stream at the end.  The staging
// buffers were allocated by the caller; the previous call on the plan is complete.
static epic_status image_host_pipelined(epic_plan_t p, const uint8_t* volt_host, int T, cudaStream_t s,
                                        float* out_host, unsigned flags)
{
    const int groups = (p->C + p->tc.cg - 1) / p->tc.cg;
    cudaError_t e = cudaSuccess;
    if (!p->copy_stream) e = cudaStreamCreateWithFlags(&p->copy_stream, cudaStreamNonBlocking);
    while (e == cudaSuccess && p->copy_ev.size() < 2 * (size_t)groups + 1) {
        cudaEvent_t ev = nullptr;
        e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        if (e == cudaSuccess) p->copy_ev.push_back(ev);
    }
    if (e != cudaSuccess) return epic::cuda_fail(p, e, "copy stream / events (host call)");
    cudaStream_t cs = p->copy_stream;
    const size_t fb = (size_t)p->A * p->P * (p->bits / 4);                   // one channel's frame
    const size_t row = (size_t)p->C * fb;                                     // one time sample
    const size_t ib = sizeof(float) * (size_t)p->nprod * p->N * p->N;         // one channel's images
    int g = 0;
    for (int c0 = 0; c0 < p->C && e == cudaSuccess; c0 += p->tc.cg, ++g) {  // every group's voltages
        const int ng = std::min(p->tc.cg, p->C - c0);
        e = cudaMemcpy2DAsync(p->stage_volt + c0 * fb, row, volt_host + c0 * fb, row, ng * fb, T,
                              cudaMemcpyHostToDevice, cs);
        if (e == cudaSuccess) e = cudaEventRecord(p->copy_ev[2 * g], cs);
    }
    if (e != cudaSuccess) return epic::cuda_fail(p, e, "cudaMemcpy2DAsync(H2D, host call)");
    int gb = 0, ga = 0;
    epic::GroupHooks hooks;
    hooks.before = [&](int, int) {
        const cudaError_t we = cudaStreamWaitEvent(s, p->copy_ev[2 * gb++], 0);
        return we == cudaSuccess ? EPIC_OK : epic::cuda_fail(p, we, "cudaStreamWaitEvent(host call)");
    };
    hooks.after = [&](int c0, int ng) {
        cudaEvent_t done = p->copy_ev[2 * ga++ + 1];
        cudaError_t ae = cudaEventRecord(done, s);
        if (ae == cudaSuccess) ae = cudaStreamWaitEvent(cs, done, 0);
        if (ae == cudaSuccess)
            ae = cudaMemcpyAsync(reinterpret_cast<uint8_t*>(out_host) + c0 * ib,
                                 reinterpret_cast<uint8_t*>(p->stage_out) + c0 * ib, ng * ib,
                                 cudaMemcpyDeviceToHost, cs);
        return ae == cudaSuccess ? EPIC_OK : epic::cuda_fail(p, ae, "cudaMemcpyAsync(D2H, host call)");
    };
    epic_status st = epic::image_run(p, p->stage_volt, T, s, p->stage_out, flags & ~EPIC_GRAPH, &hooks);
    e = cudaEventRecord(p->copy_ev[2 * groups], cs);  // the call's stream ends after the copies
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, p->copy_ev[2 * groups], 0);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (st != EPIC_OK) return st;
    if (e != cudaSuccess) return epic::cuda_fail(p, e, "cudaStreamSynchronize");
    return take_timeout(p);
}

epic_status epic_image_host(epic_plan_t p, const uint8_t* volt_host, int T, void* stream, float* out_host,
                            unsigned flags)
{
    if (!p) return EPIC_ERR_INVALID_ARG;
    if (T < 0 || T > p->max_time || !out_host || (T > 0 && !volt_host) || (p->sub > 0 && T % p->sub != 0)) {
        p->last_error = "bad T (0..max_time, a multiple of sub_int) or NULL host pointer";
        return EPIC_ERR_INVALID_ARG;
    }
    if (flags & ~(EPIC_ACCUMULATE | EPIC_TIME_KERNELS | EPIC_GRAPH)) {
        p->last_error = "unknown flag bits";
        return EPIC_ERR_INVALID_ARG;
    }
    cudaStream_t s = (cudaStream_t)stream;
    const size_t vb = (size_t)p->max_time * p->C * p->A * p->P * (p->bits / 4);
    const size_t sets_max = p->sub > 0 ? (size_t)(p->max_time / p->sub) : 1;
    const size_t set_bytes = sizeof(float) * (size_t)p->C * p->nprod * p->N * p->N;
    const size_t ob_max = std::max<size_t>(1, sets_max) * set_bytes;
    const size_t ob = (p->sub > 0 ? (size_t)(T / p->sub) : 1) * set_bytes;  // this call's image sets
    if (!p->stage_volt) {
        cudaError_t e = cudaMalloc(&p->stage_volt, vb);
        if (e == cudaSuccess) e = cudaMalloc(&p->stage_out, ob_max);
        if (e != cudaSuccess) {
            cudaFree(p->stage_volt);
            p->stage_volt = nullptr;
            return epic::cuda_fail(p, e, "cudaMalloc(host-call staging)");
        }
        p->stage_bytes = vb + ob_max;
    }
    if (p->path == EPIC_PATH_DFTGEMM_FP16 && p->sub == 0 && !(flags & EPIC_ACCUMULATE) && T > 0 && p->tc.cg < p->C)
        return image_host_pipelined(p, volt_host, T, s, out_host, flags);
    const size_t tb = (size_t)T * p->C * p->A * p->P * (p->bits / 4);
    cudaError_t e = cudaSuccess;
    if (tb) e = cudaMemcpyAsync(p->stage_volt, volt_host, tb, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && (flags & EPIC_ACCUMULATE))
        e = cudaMemcpyAsync(p->stage_out, out_host, ob, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return epic::cuda_fail(p, e, "cudaMemcpyAsync(H2D)");
    epic_status st = image_impl(p, p->stage_volt, T, s, p->stage_out, flags);
    if (st != EPIC_OK) return st;
    e = cudaMemcpyAsync(out_host, p->stage_out, ob, cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return epic::cuda_fail(p, e, "cudaMemcpyAsync(D2H)");
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return epic::cuda_fail(p, e, "cudaStreamSynchronize");
    return take_timeout(p);  // the call is complete: report (and clear) a bounded wait that ran out
}

epic_status epic_sync(epic_plan_t p)
{
    if (!p) return EPIC_ERR_INVALID_ARG;
    cudaError_t e = cudaStreamSynchronize(p->last_stream);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) return epic::cuda_fail(p, e, "epic_sync");
    return take_timeout(p);
}

epic_status epic_kernel_times(epic_plan_t p, const char** names, float* ms, int max, int* n_out)
{
    if (!p || !n_out || max < 0) return EPIC_ERR_INVALID_ARG;
    *n_out = (int)p->n_events;
    for (size_t i = 0; i < p->n_events && (int)i < max; ++i) {
        cudaError_t e = cudaEventSynchronize(p->events[i].stop);
        if (e != cudaSuccess) return epic::cuda_fail(p, e, "cudaEventSynchronize");
        float t = 0.f;
        e = cudaEventElapsedTime(&t, p->events[i].start, p->events[i].stop);
        if (e != cudaSuccess) return epic::cuda_fail(p, e, "cudaEventElapsedTime");
        if (names) names[i] = p->events[i].name;
        if (ms) ms[i] = t;
    }
    return EPIC_OK;
}

}  // extern "C"
