// C ABI of the lbem library: handle lifecycle, problem set-up, time stepping,
// outputs, diagnostics, checkpoint/resume and launch-shape autotuning.
// Every entry point is declared and documented in include/lbem.h.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "lbem_internal.cuh"

namespace lbk {

static thread_local std::string g_err;

lbem_status fail(lbem_status s, const std::string &msg) {
    g_err = msg;
    return s;
}

lbem_status cuda_fail(cudaError_t e, const char *what) {
    g_err = std::string(what) + ": " + cudaGetErrorString(e);
    return LBEM_ERR_CUDA;
}

// Guard bands: GUARD bytes of GUARD_BYTE before and after each handle-owned array, so that a kernel writing
// outside its array is caught by lbem_check_guards without a device-side checker.
constexpr size_t GUARD = 256;
constexpr unsigned char GUARD_BYTE = 0xA5;

cudaError_t gmalloc(lbem_t *h, void **p, size_t bytes, const char *name) {
    char *base = nullptr;
    *p = nullptr;
    cudaError_t e = cudaMalloc((void **)&base, bytes + 2 * GUARD);
    if (e != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(base, GUARD_BYTE, GUARD, h->stream)) != cudaSuccess ||
        (e = cudaMemsetAsync(base + GUARD + bytes, GUARD_BYTE, GUARD, h->stream)) != cudaSuccess) {
        cudaFree(base);
        return e;
    }
    *p = base + GUARD;
    h->guarded.push_back({*p, bytes, name});
    return cudaSuccess;
}

void gfree(lbem_t *h, void *p) {
    if (!p) return;
    for (size_t i = 0; i < h->guarded.size(); i++)
        if (h->guarded[i].user == p) {
            h->guarded.erase(h->guarded.begin() + i);
            break;
        }
    cudaFree(static_cast<char *>(p) - GUARD);
}

bool is_device_ptr(const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Device staging area of at least `floats` floats (grown on demand, owned by the handle).
lbem_status ensure_stage(lbem_t *h, size_t floats) {
    const size_t bytes = floats * sizeof(float);
    if (h->stage_bytes >= bytes) return LBEM_OK;
    if (h->d_stage) {
        cudaStreamSynchronize(h->stream);
        gfree(h, h->d_stage);
        h->d_stage = nullptr;
        h->stage_bytes = 0;
    }
    if (gmalloc(h, (void **)&h->d_stage, bytes, "staging") != cudaSuccess) {
        cudaGetLastError();
        return fail(LBEM_ERR_NOMEM, "staging buffer allocation failed");
    }
    h->stage_bytes = bytes;
    return LBEM_OK;
}

// A device view of caller input `p` (count floats): p itself if it is device
// memory, else a copy in the staging area at float offset `off`.
lbem_status device_input(lbem_t *h, const float *p, size_t count, size_t off, const float **out) {
    if (!p) {
        *out = nullptr;
        return LBEM_OK;
    }
    if (is_device_ptr(p)) {
        *out = p;
        return LBEM_OK;
    }
    lbem_status st = ensure_stage(h, off + count);
    if (st != LBEM_OK) return st;
    LBEM_CUDA(cudaMemcpyAsync(h->d_stage + off, p, count * sizeof(float), cudaMemcpyHostToDevice, h->stream));
    *out = h->d_stage + off;
    return LBEM_OK;
}

StepArgs step_args(const lbem_t *h, int cur_in) {
    StepArgs a;
    a.g = h->grid;
    a.in = h->buf[cur_in];
    a.out = h->buf[cur_in ^ 1];
    a.med.cL2 = h->cL2;
    a.med.mu = h->has_mu ? h->mu : nullptr;
    a.med.dlnmu = h->has_mu ? h->dlnmu : nullptr;
    a.med.ar = h->aniso_r;
    a.med.amu = h->aniso_mu;
    if (h->disp) {
        a.med.wp2 = h->d_wp2;
        a.med.wr2 = h->d_wr2;
        a.med.gam = h->d_gam;
        a.med.pc = h->d_pc;
        a.med.pb = h->d_pb;
        a.med.pa = h->d_pa;
        a.med.J = h->d_J;
        a.med.Pr = h->pole_P(cur_in);
        a.med.Pw = h->pole_P(cur_in ^ 1);
    }
    a.evt.rowptr = h->nev ? h->d_rowptr : nullptr;
    a.evt.ev = h->d_ev;
    a.evt.amp = h->d_amp;
    a.evt.nt = h->nsrc ? h->nt : 0;
    a.evt.traces = h->d_traces;
    a.evt.cap = h->nrec ? h->cap : 0;
    a.t = h->t;
    a.sched = reinterpret_cast<int *>(h->d_counter) + 2;
    return a;
}

static Walls handle_walls(const lbem_t *h) {
    Walls w;
    for (int a = 0; a < 3; a++) w.kind[a] = h->bc[a];
    w.fx = h->bc[0] ? h->d_fx : nullptr;
    w.fy = h->bc[1] ? h->d_fy : nullptr;
    w.fz = h->bc[2] ? h->d_fz : nullptr;
    return w;
}

static cudaError_t launch_step(const lbem_t *h, const StepArgs &a, int variant) {
    if (h->general()) {
        General q;
        if (h->disp) {
            q.wp2 = h->d_wp2;
            q.wr2 = h->d_wr2;
            q.gam = h->d_gam;
            q.pc = h->d_pc;
            q.pb = h->d_pb;
            q.pa = h->d_pa;
            q.J = h->d_J;
            q.P = a.med.Pr;
            q.Pn = a.med.Pw;
        }
        q.r = h->aniso_r;
        q.mubar = h->aniso_mu;
        return launch_step_2d_gen(a, handle_walls(h), q, h->stream);
    }
    if (h->dim == 2) return launch_step_2d(a, h->storage, h->has_mu, variant, h->stream);
    const Walls w = handle_walls(h);
    return launch_step_3d(a, h->has_mu, variant, h->stream, &w);  // walls and layers applied in the kernel
}

static int two_step_shape(const lbem_t *h);
// what a captured graph depends on besides t, nsteps and the buffer: kernel variant and two-step shape
static int graph_key(const lbem_t *h) { return (h->variant * 4 + h->tblock) * 16 + two_step_shape(h) + 1; }

// Whether launches of two (three) steps apply: 2D; FP32 storage with any medium, 16-bit storage with uniform mu
// and nx % 4 == 0; three steps per launch exist for FP32 storage with uniform mu.
// An anisotropic medium or a dispersive pole takes two steps per launch unless a heterogeneous mu comes with it,
// or walls with the pole, which the general single-step kernel handles (with walls an anisotropic medium's launches
// of two steps are followed by the anisotropic edge pass).
static bool multi_step_base(const lbem_t *h) {
    if (h->general() && (h->has_mu || (h->walls() && h->disp))) return false;
    return h->dim == 2 && (h->storage == LBEM_F32 || (!h->has_mu && h->grid.nx % 4 == 0));
}
static bool two_step_ok(const lbem_t *h) { return h->tblock >= 2 && multi_step_base(h); }
static bool three_step_ok(const lbem_t *h) {
    return h->tblock == 3 && multi_step_base(h) && h->storage == LBEM_F32 && !h->has_mu && !h->general();
}
// Two-step shapes of the handle's medium: a dispersive pole 1 (the tile kernel), an anisotropic tensor 2 (the tile
// kernel, the strip kernel), otherwise those of tblock.cu.
static int two_step_nshapes(const lbem_t *h) {
    return h->disp ? 1 : h->aniso ? 2 : tb2_nshapes(h->storage, h->has_mu);
}
// The two-step shape to launch: the one set (or autotuned) when it exists for this medium, else 0, except that a
// large FP32 grid (at least 12M sites) without a pole defaults to the strip-streaming kernel (sstream.cu; uniform mu
// at 4096^2: 274.6k Mlups against 247.3k for tile shape 0; at 2048^2 and below the tile kernel is faster): shape 10
// for uniform mu, 2 with a heterogeneous mu, 1 with an anisotropic tensor.
static int two_step_shape(const lbem_t *h) {
    if (h->disp) return 0;
    const bool big = h->tblock == 2 && h->dim == 2 && h->storage == LBEM_F32 && h->nsite >= 12000000;
    if (h->aniso) return h->tb_shape_set ? (h->tb_shape == 1 ? 1 : 0) : (big ? 1 : 0);
    if (!h->tb_shape_set && big) return h->has_mu ? 2 : 7 + rs2_nshapes() + 1;
    return h->tblock == 2 && h->tb_shape < tb2_nshapes(h->storage, h->has_mu) ? h->tb_shape : 0;
}
static int steps_per_launch(const lbem_t *h) { return three_step_ok(h) ? 3 : two_step_ok(h) ? 2 : 1; }

// Enqueue nsteps steps starting from buffer `cur` at time t0: triples (pairs) of steps with the three-step
// (two-step) kernel when enabled, a remaining pair with the two-step kernel's default tile, single steps
// otherwise; returns the buffer holding the final state in *cur_out.
// With walls: the k steps of a launch recomputed on the bands the walls and layers change (walls.cu); the
// general kernel's single steps apply walls and layers themselves (a pole with walls steps only that way).
static cudaError_t edge_fixup(const lbem_t *h, const StepArgs &a, int k, cudaStream_t s) {
    if (!h->walls() || h->dim != 2 || h->disp || (h->aniso && k == 1)) return cudaSuccess;
    return launch_edge_2d(a, handle_walls(h), h->d_tiles[k], h->ntiles[k],
                          h->has_mu ? h->tile_smem_mu[k] : h->tile_smem[k], k, h->aniso, s);
}
static cudaError_t edge_fixup(const lbem_t *h, const StepArgs &a, int k) { return edge_fixup(h, a, k, h->stream); }

// Whether a two-step shape is a strip-streaming launch (sstream.cu) for this medium.
static bool strip_shape(const lbem_t *h, int shape) {
    if (h->storage != LBEM_F32 || h->disp) return false;
    const int first = 7 + rs2_nshapes();  // the strip shapes follow the tile and register-streaming ones
    return h->aniso ? shape == 1 : h->has_mu ? shape == 2 : shape >= first && shape < first + ss2_nshapes();
}

// With walls, a strip-streaming launch of k steps writes only outside the bands the edge pass rewrites (the edge
// tiles' bands: the sites within max(L, 1) + k - 1 of a wall, the whole axis when the two bands meet), so that the
// two launches write disjoint sites and the edge pass can run beside it.
static void write_window(const lbem_t *h, int k, StepArgs &a) {
    const int bw = std::max(h->layer, 1) + k - 1, n[2] = {h->grid.nx, h->grid.ny};
    int *lo[2] = {&a.wx0, &a.wy0}, *hi[2] = {&a.wx1, &a.wy1};
    for (int d = 0; d < 2; d++) {
        if (!h->bc[d]) continue;
        const bool all = 2 * bw >= n[d];
        *lo[d] = all ? 0 : bw;
        *hi[d] = all ? 0 : n[d] - bw;
    }
}

static cudaError_t enqueue_steps(const lbem_t *h, int cur, long long t0, int nsteps, int *cur_out) {
    int n = 0;
    if (three_step_ok(h)) {
        for (; n + 3 <= nsteps; n += 3) {
            StepArgs a = step_args(h, cur);
            a.t = t0 + n;
            cudaError_t e = launch_step_2d_tb3(a, h->tb_shape, h->stream);
            if (e == cudaSuccess) e = edge_fixup(h, a, 3);
            if (e != cudaSuccess) return e;
            cur ^= 1;
        }
    }
    if (two_step_ok(h)) {
        const int shape = two_step_shape(h);
        // walls beside a strip-streaming launch: fork the edge pass onto its stream, launch it first (its tiles
        // take their SMs before the persistent strip grid fills them), and join it before the next launch
        const bool beside = h->walls() && h->dim == 2 && h->edge_stream && strip_shape(h, shape);
        for (; n + 2 <= nsteps; n += 2) {
            StepArgs a = step_args(h, cur);
            a.t = t0 + n;
            cudaError_t e;
            if (beside) {
                write_window(h, 2, a);
                e = cudaEventRecord(h->ev_fork, h->stream);
                if (e == cudaSuccess) e = cudaStreamWaitEvent(h->edge_stream, h->ev_fork, 0);
                if (e == cudaSuccess) e = edge_fixup(h, a, 2, h->edge_stream);
                if (e == cudaSuccess) e = cudaEventRecord(h->ev_join, h->edge_stream);
                if (e == cudaSuccess) e = launch_step_2d_tb2(a, h->storage, shape, h->stream);
                if (e == cudaSuccess) e = cudaStreamWaitEvent(h->stream, h->ev_join, 0);
            } else {
                e = launch_step_2d_tb2(a, h->storage, shape, h->stream);
                if (e == cudaSuccess) e = edge_fixup(h, a, 2);
            }
            if (e != cudaSuccess) return e;
            cur ^= 1;
        }
    }
    for (; n < nsteps; n++) {
        StepArgs a = step_args(h, cur);
        a.t = t0 + n;
        cudaError_t e = launch_step(h, a, h->variant);
        if (e == cudaSuccess) e = edge_fixup(h, a, 1);
        if (e != cudaSuccess) return e;
        cur ^= 1;
    }
    *cur_out = cur;
    return cudaSuccess;
}

static void drop_graph(lbem_t *h) {
    if (h->graph) cudaGraphExecDestroy(h->graph);
    h->graph = nullptr;
    h->graph_t0 = -1;
}

static size_t elem_bytes(int storage) { return storage == LBEM_F32 ? 4 : 2; }

static lbem_status rebuild_events(lbem_t *h) {
    std::vector<Event> ev;
    std::vector<long long> rows;
    const int nx = h->grid.nx;
    for (int k = 0; k < h->nsrc; k++) {
        ev.push_back(Event{(int)(h->src_site[k] % nx), 0, k, h->src_comp[k]});
        rows.push_back(h->src_site[k] / nx);
    }
    for (int r = 0; r < h->nrec; r++) {
        ev.push_back(Event{(int)(h->rec_site[r] % nx), 1, r, h->rec_comp[r]});
        rows.push_back(h->rec_site[r] / nx);
    }
    std::vector<int> order(ev.size());
    for (size_t i = 0; i < order.size(); i++) order[i] = (int)i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return rows[a] < rows[b]; });
    std::vector<Event> sorted(ev.size());
    std::vector<int> rowptr(h->grid.nrows + 1, 0);
    for (size_t i = 0; i < order.size(); i++) {
        sorted[i] = ev[order[i]];
        rowptr[rows[order[i]] + 1]++;
    }
    for (int r = 0; r < h->grid.nrows; r++) rowptr[r + 1] += rowptr[r];
    cudaStreamSynchronize(h->stream);
    gfree(h, h->d_ev);
    h->d_ev = nullptr;
    h->nev = (int)sorted.size();
    if (!h->d_rowptr) LBEM_CUDA(gmalloc(h, (void **)&h->d_rowptr, sizeof(int) * (h->grid.nrows + 1), "event rows"));
    LBEM_CUDA(cudaMemcpy(h->d_rowptr, rowptr.data(), sizeof(int) * rowptr.size(), cudaMemcpyHostToDevice));
    if (h->nev) {
        LBEM_CUDA(gmalloc(h, (void **)&h->d_ev, sizeof(Event) * sorted.size(), "events"));
        LBEM_CUDA(cudaMemcpy(h->d_ev, sorted.data(), sizeof(Event) * sorted.size(), cudaMemcpyHostToDevice));
    }
    drop_graph(h);
    return LBEM_OK;
}

}  // namespace lbk

using namespace lbk;

namespace lbk {

// Rows of a slab's halo (spatial domain decomposition, 2D): (row, plane) pairs, in the order the buffer holds them.
struct HaloRows {
    int n;
    int row[5], plane[5];
};

// Copy the listed rows (nx floats each) of the state to buf ([k][nx]) or back.
__global__ void halo_rows_kernel(float *state, long long plane_stride, int pitch, int nx, HaloRows spec, float *buf,
                                 int to_state) {
    const int k = blockIdx.y;
    float *r = state + spec.plane[k] * plane_stride + (long long)spec.row[k] * pitch;
    float *b = buf + (long long)k * nx;
    for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < nx; x += gridDim.x * blockDim.x) {
        if (to_state)
            r[x] = b[x];
        else
            b[x] = r[x];
    }
}

// The rows a neighbour needs (out) or that a neighbour's rows fill (in), for a slab of ny rows with `halo` ghost rows
// on either side (real rows halo .. ny - halo - 1); pull streaming: a row pulls g_2 from the row below, g_4 from
// the row above.  halo 1: g_2 of the last real row up, g_4 of the first down.  halo 2 (two steps per exchange): the
// inner ghost row's first collision feeds a real row, so it needs its own g_0, g_1, g_3 and the population it pulls
// from the outer ghost row.
static HaloRows halo_spec(int halo, int ny, bool upper, bool out) {
    HaloRows s{};
    auto add = [&](int row, int plane) {
        s.row[s.n] = row;
        s.plane[s.n] = plane;
        s.n++;
    };
    if (halo == 1) {
        if (out) add(upper ? ny - 2 : 1, upper ? 2 : 4);
        else add(upper ? ny - 1 : 0, upper ? 4 : 2);
        return s;
    }
    // out upper: last real row (ny - 3) planes 0-3, the row below it plane 2; in lower ghosts in the same order
    // out lower: first real row (2) planes 0, 1, 3, 4, the row above it plane 4; in upper ghosts in the same order
    const int r1 = out ? (upper ? ny - 3 : 2) : (upper ? ny - 2 : 1);
    const int r2 = out ? (upper ? ny - 4 : 3) : (upper ? ny - 1 : 0);
    const bool up_going = out ? upper : !upper;  // populations moving +y (sent up, received from below)
    for (int p : {0, 1, up_going ? 2 : 3, up_going ? 3 : 4}) add(r1, p);
    add(r2, up_going ? 2 : 4);
    return s;
}

}  // namespace lbk

extern "C" {

const char *lbem_last_error(void) { return g_err.c_str(); }

lbem_status lbem_create(const lbem_desc *d, lbem_t **out) {
    if (!d || !out) return fail(LBEM_ERR_ARG, "lbem_create: null argument");
    *out = nullptr;
    if (d->dim != 2 && d->dim != 3) return fail(LBEM_ERR_ARG, "lbem_create: dim must be 2 or 3");
    const int nz = d->dim == 3 ? d->nz : 1;
    if (d->nx < 1 || d->ny < 1 || nz < 1) return fail(LBEM_ERR_ARG, "lbem_create: grid sizes must be >= 1");
    if (d->storage < LBEM_F32 || d->storage > LBEM_I16B) return fail(LBEM_ERR_ARG, "lbem_create: unknown storage");
    if (d->dim == 3 && d->storage != LBEM_F32) return fail(LBEM_ERR_ARG, "lbem_create: 3D supports LBEM_F32 storage only");
    if (d->nx > (1 << 28) || (long long)d->ny * nz > (1LL << 30))
        return fail(LBEM_ERR_ARG, "lbem_create: grid too large");
    lbem_t *h = new lbem_t();
    h->dim = d->dim;
    h->storage = d->storage;
    h->npop = d->dim == 2 ? 5 : 21;
    h->c_ref2 = d->c_ref2 > 0 ? d->c_ref2 : (d->dim == 2 ? 0.5 : 1.0 / 6.0);
    h->stream = (cudaStream_t)d->stream;
    // default launch shape: the fastest measured on GB300 for each form (lbem_autotune re-measures)
    h->variant = d->dim == 3 ? 1 : (d->storage == LBEM_F32 ? 0 : 6);
    Grid &G = h->grid;
    G.nx = d->nx;
    G.ny = d->ny;
    G.nz = nz;
    G.nrows = d->ny * nz;
    G.nchunk = (d->nx + 3) / 4;
    G.nchunk_pad = round_up(G.nchunk, 32);
    G.pitch = round_up(d->nx, 32);  // 128-byte aligned FP32 rows; >= 4 * nchunk
    G.plane = (long long)G.pitch * G.nrows;
    h->nsite = (long long)d->nx * d->ny * nz;
    const size_t eb = elem_bytes(h->storage);
    const size_t data_bytes = (size_t)h->npop * G.plane * eb;
    const size_t ex_bytes = h->storage == LBEM_I16B ? (size_t)h->npop * (G.pitch / 4) * G.nrows : 0;
    const size_t per = ((data_bytes + 255) / 256 * 256) + ((ex_bytes + 255) / 256 * 256);
    h->pool_bytes = 2 * per;
    cudaError_t e = gmalloc(h, &h->pool, h->pool_bytes, "populations");
    if (e == cudaSuccess) e = gmalloc(h, (void **)&h->cL2, sizeof(float) * G.plane, "c_L^2");
    if (e == cudaSuccess) {
        h->n_partials = diag_blocks(h->nsite);
        e = gmalloc(h, (void **)&h->d_partials, sizeof(double) * 3 * h->n_partials, "diagnostic partials");
    }
    if (e == cudaSuccess) e = gmalloc(h, (void **)&h->d_diag, sizeof(double) * 4, "diagnostics");
    if (e == cudaSuccess) e = gmalloc(h, (void **)&h->d_counter, sizeof(unsigned) * 4, "counters");  // [2..3]: StepArgs::sched
    if (e != cudaSuccess) {
        cudaGetLastError();
        lbem_destroy(h);
        return fail(LBEM_ERR_NOMEM, "lbem_create: device allocation failed");
    }
    for (int b = 0; b < 2; b++) {
        PopBuf &p = h->buf[b];
        char *base = (char *)h->pool + b * per;
        p.data = base;
        p.ex = ex_bytes ? (int8_t *)(base + (data_bytes + 255) / 256 * 256) : nullptr;
        p.plane = G.plane;
        p.pitch = G.pitch;
        p.expitch = G.pitch / 4;
        p.explane = (long long)(G.pitch / 4) * G.nrows;
        p.scale = p.inv_scale = 1.f;
    }
    cudaMemsetAsync(h->pool, 0, h->pool_bytes, h->stream);
    cudaMemsetAsync(h->cL2, 0, sizeof(float) * G.plane, h->stream);
    cudaMemsetAsync(h->d_counter, 0, sizeof(unsigned) * 4, h->stream);
    if ((e = cudaStreamSynchronize(h->stream)) != cudaSuccess) {
        lbem_destroy(h);
        return cuda_fail(e, "lbem_create");
    }
    *out = h;
    return LBEM_OK;
}

void lbem_destroy(lbem_t *h) {
    if (!h) return;
    cudaStreamSynchronize(h->stream);
    drop_graph(h);
    adjoint_free(h);
    for (void *p : {(void *)h->pool, (void *)h->cL2, (void *)h->mu, (void *)h->dlnmu, (void *)h->d_rowptr,
                    (void *)h->d_ev, (void *)h->d_amp, (void *)h->d_traces, (void *)h->d_partials,
                    (void *)h->d_diag, (void *)h->d_counter, (void *)h->d_stage, (void *)h->d_fx, (void *)h->d_fy,
                    (void *)h->d_fz,
                    (void *)h->d_wp2, (void *)h->d_wr2, (void *)h->d_gam, (void *)h->d_J, (void *)h->d_P,
                    (void *)h->d_P2, (void *)h->d_pc, (void *)h->d_pb, (void *)h->d_pa})
        gfree(h, p);
    for (int k = 1; k <= 3; k++) gfree(h, h->d_tiles[k]);
    if (h->edge_stream) {
        cudaStreamSynchronize(h->edge_stream);
        cudaStreamDestroy(h->edge_stream);
    }
    if (h->ev_fork) cudaEventDestroy(h->ev_fork);
    if (h->ev_join) cudaEventDestroy(h->ev_join);
    delete h;
}

lbem_status lbem_set_stream(lbem_t *h, void *stream) {
    if (!h) return fail(LBEM_ERR_ARG, "null handle");
    cudaStreamSynchronize(h->stream);
    h->stream = (cudaStream_t)stream;
    drop_graph(h);
    return LBEM_OK;
}

lbem_status lbem_sync(lbem_t *h) {
    if (!h) return fail(LBEM_ERR_ARG, "null handle");
    LBEM_CUDA(cudaStreamSynchronize(h->stream));
    LBEM_CUDA(cudaGetLastError());
    if (tb2_take_timeouts())
        return fail(LBEM_ERR_TIMEOUT, "lbem_sync: a tile load of the multi-step kernel did not complete within the wait limit");
    return LBEM_OK;
}

lbem_status lbem_set_wait_limit(double seconds) {
    if (!(seconds >= 0.0 && seconds <= 3600.0)) return fail(LBEM_ERR_ARG, "lbem_set_wait_limit: seconds must lie in [0, 3600]");
    LBEM_CUDA(tb_set_wait_limit((unsigned long long)(seconds * 1e9)));
    return LBEM_OK;
}

lbem_status lbem_info(const lbem_t *h, long long *nsite, size_t *state_bytes) {
    if (!h) return fail(LBEM_ERR_ARG, "null handle");
    if (nsite) *nsite = h->nsite;
    if (state_bytes) {
        size_t b = (size_t)h->npop * h->grid.plane * elem_bytes(h->storage);
        if (h->storage == LBEM_I16B) b += (size_t)h->npop * h->buf[0].explane;
        if (h->disp) b += 2 * sizeof(float) * (size_t)h->grid.plane;  // the pole's J and P planes
        *state_bytes = b;
    }
    return LBEM_OK;
}

// Medium upload shared by lbem_set_medium (isotropic, mu_r per site or NULL) and lbem_set_medium_aniso (a
// uniform in-plane tensor diag(mu_xx, mu_yy), mu_r NULL): validate everything first, then write.
static lbem_status set_medium(lbem_t *h, const float *eps_r, const float *mu_r, bool aniso, double mu_xx,
                              double mu_yy, const char *who) {
    const std::string name(who);
    const float *de, *dm;
    lbem_status st = device_input(h, eps_r, h->nsite, 0, &de);
    if (st != LBEM_OK) return st;
    if ((st = device_input(h, mu_r, h->nsite, h->nsite, &dm)) != LBEM_OK) return st;
    const double r = aniso ? sqrt(mu_xx / mu_yy) : 1.0, mubar = aniso ? sqrt(mu_xx * mu_yy) : 1.0;
    const double fsum = aniso ? (double)((float)r + 1.f / (float)r) : (double)h->dim;
    LBEM_CUDA(launch_medium(h, de, dm, fsum, mubar, h->d_counter, h->stream));
    unsigned bad = 0;
    LBEM_CUDA(cudaMemcpyAsync(&bad, h->d_counter, sizeof(unsigned), cudaMemcpyDeviceToHost, h->stream));
    LBEM_CUDA(cudaStreamSynchronize(h->stream));
    if (bad)
        return fail(LBEM_ERR_MEDIUM, name + ": " + std::to_string(bad) +
                                         " sites with eps_r or mu_r not finite and > 0, or rest weight w0 outside "
                                         "[0,1) (medium faster than c_ref)");
    if (h->disp) {  // the pole must stay within its stability bound in the new medium
        LBEM_CUDA(cudaMemsetAsync(h->d_counter, 0, sizeof(unsigned), h->stream));
        LBEM_CUDA(launch_disp_check(h, de, dm, fsum, mubar, h->d_wp2, h->d_wr2, h->d_gam, true, h->d_counter,
                                    h->stream));
        LBEM_CUDA(cudaMemcpyAsync(&bad, h->d_counter, sizeof(unsigned), cudaMemcpyDeviceToHost, h->stream));
        LBEM_CUDA(cudaStreamSynchronize(h->stream));
        if (bad)
            return fail(LBEM_ERR_MEDIUM, name + ": " + std::to_string(bad) +
                                             " sites where the dispersive pole exceeds wp^2 + wr^2 <= 4 w0");
    }
    if (dm && !h->mu) {
        LBEM_CUDA(gmalloc(h, (void **)&h->mu, sizeof(float) * h->grid.plane, "mu"));
        LBEM_CUDA(gmalloc(h, (void **)&h->dlnmu, sizeof(float) * h->grid.plane * h->dim, "grad ln mu"));
        LBEM_CUDA(cudaMemsetAsync(h->mu, 0, sizeof(float) * h->grid.plane, h->stream));
        LBEM_CUDA(cudaMemsetAsync(h->dlnmu, 0, sizeof(float) * h->grid.plane * h->dim, h->stream));
    }
    LBEM_CUDA(launch_medium_write(h, de, dm, mubar, h->stream));
    if (dm && h->walls()) LBEM_CUDA(launch_medium_grad_walls(h, h->stream));
    h->has_mu = dm != nullptr;
    h->aniso = aniso;
    h->aniso_r = (float)r;
    h->aniso_mu = (float)mubar;
    h->has_medium = true;
    drop_graph(h);
    return LBEM_OK;
}

lbem_status lbem_set_medium(lbem_t *h, const float *eps_r, const float *mu_r) {
    if (!h || !eps_r) return fail(LBEM_ERR_ARG, "lbem_set_medium: null argument");
    return set_medium(h, eps_r, mu_r, false, 1.0, 1.0, "lbem_set_medium");
}

lbem_status lbem_set_medium_aniso(lbem_t *h, const float *eps_r, double mu_xx, double mu_yy) {
    if (!h || !eps_r) return fail(LBEM_ERR_ARG, "lbem_set_medium_aniso: null argument");
    if (h->dim != 2 || h->storage != LBEM_F32)
        return fail(LBEM_ERR_ARG, "lbem_set_medium_aniso: 2D grids with LBEM_F32 storage only");
    if (!(mu_xx > 0.0 && mu_yy > 0.0 && isfinite(mu_xx) && isfinite(mu_yy)))
        return fail(LBEM_ERR_ARG, "lbem_set_medium_aniso: mu_xx and mu_yy must be finite and > 0");
    if (h->adj) return fail(LBEM_ERR_STATE, "lbem_set_medium_aniso: a recorded adjoint run exists (isotropic only)");
    return set_medium(h, eps_r, nullptr, true, mu_xx, mu_yy, "lbem_set_medium_aniso");
}

lbem_status lbem_set_fields(lbem_t *h, const float *E, const float *B) {
    if (!h) return fail(LBEM_ERR_ARG, "null handle");
    if (!h->has_medium) return fail(LBEM_ERR_STATE, "lbem_set_fields: set a medium first");
    const size_t n3 = 3 * (size_t)h->nsite;
    const float *dE, *dB;
    lbem_status st = device_input(h, E, n3, 0, &dE);
    if (st != LBEM_OK) return st;
    if ((st = device_input(h, B, n3, n3, &dB)) != LBEM_OK) return st;
    if (h->storage == LBEM_F16) {
        // power-of-two scale mapping the largest input magnitude to ~2^7 (headroom ~2^9 below the
        // binary16 maximum for the populations, which can exceed the fields by the factor w0/c_L^2)
        LBEM_CUDA(cudaMemsetAsync(h->d_counter, 0, sizeof(unsigned), h->stream));
        if (dE) LBEM_CUDA(launch_maxabs(dE, n3, h->d_counter, h->stream));
        if (dB) LBEM_CUDA(launch_maxabs(dB, n3, h->d_counter, h->stream));
        unsigned bits = 0;
        LBEM_CUDA(cudaMemcpyAsync(&bits, h->d_counter, sizeof(unsigned), cudaMemcpyDeviceToHost, h->stream));
        LBEM_CUDA(cudaStreamSynchronize(h->stream));
        float m;
        memcpy(&m, &bits, sizeof(m));
        for (float a : h->src_amp) m = fmaxf(m, fabsf(a));
        int k = 0;
        if (m > 0 && isfinite(m)) k = 7 - (int)ceil(log2((double)m));
        k = std::max(-40, std::min(40, k));
        const float s = ldexpf(1.f, k);
        for (int b = 0; b < 2; b++) {
            h->buf[b].scale = s;
            h->buf[b].inv_scale = 1.f / s;
        }
    }
    cudaError_t e = h->dim == 2 ? launch_init_2d(h, dE, dB, h->stream) : launch_init_3d(h, dE, dB, h->stream);
    LBEM_CUDA(e);
    h->t = 0;
    h->wd_last = -1.0;
    if (h->d_traces) LBEM_CUDA(cudaMemsetAsync(h->d_traces, 0, sizeof(float) * (size_t)h->nrec * h->cap, h->stream));
    if (h->disp) {  // the pole starts at rest: D = E
        for (float *p : {h->d_J, h->d_P, h->d_P2})
            LBEM_CUDA(cudaMemsetAsync(p, 0, sizeof(float) * (size_t)h->grid.plane, h->stream));
    }
    drop_graph(h);
    return LBEM_OK;
}

lbem_status lbem_set_sources(lbem_t *h, int n, const long long *site, const int *comp, const float *amp, int nt) {
    if (!h) return fail(LBEM_ERR_ARG, "null handle");
    if (n < 0 || n > 65536) return fail(LBEM_ERR_ARG, "lbem_set_sources: 0 <= n <= 65536");
    if (n > 0 && (!site || !comp || !amp || nt < 1)) return fail(LBEM_ERR_ARG, "lbem_set_sources: null array or nt < 1");
    for (int k = 0; k < n; k++) {
        if (site[k] < 0 || site[k] >= h->nsite) return fail(LBEM_ERR_ARG, "lbem_set_sources: site out of range");
        if (comp[k] < 0 || comp[k] > 2) return fail(LBEM_ERR_ARG, "lbem_set_sources: comp must be 0..2");
    }
    h->src_site.assign(site, site + n);
    h->src_comp.assign(comp, comp + n);
    h->src_amp.assign(amp, amp + (size_t)n * (n ? nt : 0));
    h->nsrc = n;
    h->nt = n ? nt : 0;
    cudaStreamSynchronize(h->stream);
    gfree(h, h->d_amp);
    h->d_amp = nullptr;
    if (n) {
        LBEM_CUDA(gmalloc(h, (void **)&h->d_amp, sizeof(float) * (size_t)n * nt, "source amplitudes"));
        LBEM_CUDA(cudaMemcpy(h->d_amp, amp, sizeof(float) * (size_t)n * nt, cudaMemcpyHostToDevice));
    }
    return rebuild_events(h);
}

lbem_status lbem_set_receivers(lbem_t *h, int n, const long long *site, const int *comp, int capacity) {
    if (!h) return fail(LBEM_ERR_ARG, "null handle");
    if (n < 0 || n > 65536 || capacity < 0) return fail(LBEM_ERR_ARG, "lbem_set_receivers: 0 <= n <= 65536, capacity >= 0");
    if (n > 0 && (!site || !comp)) return fail(LBEM_ERR_ARG, "lbem_set_receivers: null array");
    for (int r = 0; r < n; r++) {
        if (site[r] < 0 || site[r] >= h->nsite) return fail(LBEM_ERR_ARG, "lbem_set_receivers: site out of range");
        if (comp[r] < 0 || comp[r] > 5) return fail(LBEM_ERR_ARG, "lbem_set_receivers: comp must be 0..5");
    }
    h->rec_site.assign(site, site + n);
    h->rec_comp.assign(comp, comp + n);
    h->nrec = n;
    h->cap = capacity;
    cudaStreamSynchronize(h->stream);
    gfree(h, h->d_traces);
    h->d_traces = nullptr;
    if (n && capacity) {
        LBEM_CUDA(gmalloc(h, (void **)&h->d_traces, sizeof(float) * (size_t)n * capacity, "traces"));
        LBEM_CUDA(cudaMemset(h->d_traces, 0, sizeof(float) * (size_t)n * capacity));
    } else {
        h->cap = 0;
    }
    return rebuild_events(h);
}

lbem_status lbem_set_graphs(lbem_t *h, int on) {
    if (!h) return fail(LBEM_ERR_ARG, "null handle");
    h->use_graphs = on != 0;
    if (!on) drop_graph(h);
    return LBEM_OK;
}

static lbem_status step_run(lbem_t *h, int nsteps);

lbem_status lbem_set_watchdog(lbem_t *h, int every, double max_growth) {
    if (!h) return fail(LBEM_ERR_ARG, "null handle");
    if (every < 0 || (every > 0 && !(max_growth > 1.0)))
        return fail(LBEM_ERR_ARG, "lbem_set_watchdog: every >= 0 and max_growth > 1");
    h->wd_every = every;
    h->wd_growth = max_growth;
    h->wd_last = -1.0;
    return LBEM_OK;
}

lbem_status lbem_step(lbem_t *h, int nsteps) {
    if (!h) return fail(LBEM_ERR_ARG, "null handle");
    if (h->wd_every <= 0 || nsteps <= 0) return step_run(h, nsteps);
    // watchdog: FP64 field energy after every `wd_every` steps; non-finite or a jump by more than
    // wd_growth since the previous check stops the run
    int left = nsteps;
    while (left > 0) {
        const long long into = h->t % h->wd_every;
        const int chunk = (int)std::min<long long>(left, h->wd_every - into);
        lbem_status st = step_run(h, chunk);
        if (st != LBEM_OK) return st;
        left -= chunk;
        if ((h->t % h->wd_every) == 0) {
            double d[3];
            st = lbem_diagnostics(h, d);
            if (st == LBEM_ERR_UNSTABLE)
                return fail(LBEM_ERR_UNSTABLE, "lbem_step: watchdog found a non-finite state at t = " + std::to_string(h->t));
            if (st != LBEM_OK) return st;
            if (h->wd_last > 0.0 && d[0] > h->wd_growth * h->wd_last)
                return fail(LBEM_ERR_UNSTABLE, "lbem_step: watchdog: field energy grew by more than the allowed factor "
                                               "between checks at t = " + std::to_string(h->t));
            h->wd_last = d[0];
        }
    }
    return LBEM_OK;
}

static lbem_status step_run(lbem_t *h, int nsteps) {
    if (!h) return fail(LBEM_ERR_ARG, "null handle");
    if (nsteps < 0) return fail(LBEM_ERR_ARG, "lbem_step: nsteps < 0");
    if (!h->has_medium) return fail(LBEM_ERR_STATE, "lbem_step: set a medium first");
    if (nsteps == 0) return LBEM_OK;
    if (h->use_graphs && h->stream == nullptr)
        return fail(LBEM_ERR_STATE, "lbem_step: CUDA graphs need a non-default stream (lbem_set_stream)");
    if (h->use_graphs) {
        if (!(h->graph && h->graph_t0 == h->t && h->graph_steps == nsteps && h->graph_cur == h->cur &&
              h->graph_variant == graph_key(h))) {
            drop_graph(h);
            LBEM_CUDA(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
            int cur_end = h->cur;
            cudaError_t e = enqueue_steps(h, h->cur, h->t, nsteps, &cur_end);
            if (e != cudaSuccess) {
                cudaGraph_t g = nullptr;
                cudaStreamEndCapture(h->stream, &g);
                if (g) cudaGraphDestroy(g);
                return cuda_fail(e, "lbem_step (capture)");
            }
            h->graph_cur_end = cur_end;
            cudaGraph_t g = nullptr;
            LBEM_CUDA(cudaStreamEndCapture(h->stream, &g));
            e = cudaGraphInstantiate(&h->graph, g, 0);
            cudaGraphDestroy(g);
            LBEM_CUDA(e);
            h->graph_t0 = h->t;
            h->graph_steps = nsteps;
            h->graph_cur = h->cur;
            h->graph_variant = graph_key(h);
        }
        LBEM_CUDA(cudaGraphLaunch(h->graph, h->stream));
        h->cur = h->graph_cur_end;
        h->t += nsteps;
        return LBEM_OK;
    }
    int cur_end = h->cur;
    LBEM_CUDA(enqueue_steps(h, h->cur, h->t, nsteps, &cur_end));
    h->cur = cur_end;
    h->t += nsteps;
    return LBEM_OK;
}

lbem_status lbem_set_temporal_blocking(lbem_t *h, int steps_per_pass, int tile_shape) {
    if (!h) return fail(LBEM_ERR_ARG, "null handle");
    if (steps_per_pass < 1 || steps_per_pass > 3)
        return fail(LBEM_ERR_ARG, "lbem_set_temporal_blocking: steps_per_pass must be 1, 2 or 3");
    if (tile_shape < -1 || tile_shape >= (steps_per_pass == 3 ? tb3_nshapes() : tb2_nshapes(h->storage, h->has_mu)))
        return fail(LBEM_ERR_ARG, "lbem_set_temporal_blocking: tile_shape out of range");
    h->tblock = steps_per_pass;
    h->tb_shape = tile_shape < 0 ? 0 : tile_shape;
    h->tb_shape_set = tile_shape >= 0;
    drop_graph(h);
    return LBEM_OK;
}

lbem_status lbem_set_boundaries(lbem_t *h, const int kind[3], int layer, double gamma_max) {
    if (!h || !kind) return fail(LBEM_ERR_ARG, "null argument");
    for (int a = 0; a < 3; a++)
        if (kind[a] < LBEM_BC_PERIODIC || kind[a] > LBEM_BC_PMC)
            return fail(LBEM_ERR_ARG, "lbem_set_boundaries: kind must be LBEM_BC_PERIODIC, _PEC or _PMC");
    const bool any = kind[0] || kind[1] || kind[2];
    if (any && h->dim == 2 && kind[2]) return fail(LBEM_ERR_ARG, "lbem_set_boundaries: a 2D grid has no z walls");
    if (any && h->storage != LBEM_F32) return fail(LBEM_ERR_ARG, "lbem_set_boundaries: walls need LBEM_F32 storage");
    if (layer < 0 || !(gamma_max >= 0.0 && gamma_max < 1.0))
        return fail(LBEM_ERR_ARG, "lbem_set_boundaries: layer >= 0 and 0 <= gamma_max < 1");
    if (layer > 0 && !any) return fail(LBEM_ERR_ARG, "lbem_set_boundaries: an absorbing layer needs a wall");
    if ((kind[0] && 2 * layer > h->grid.nx) || (kind[1] && 2 * layer > h->grid.ny) ||
        (kind[2] && 2 * layer > h->grid.nz))
        return fail(LBEM_ERR_ARG, "lbem_set_boundaries: layer wider than half the walled axis");
    if (h->adj) return fail(LBEM_ERR_STATE, "lbem_set_boundaries: a recorded adjoint run exists (periodic only)");
    LBEM_CUDA(cudaStreamSynchronize(h->stream));
    gfree(h, h->d_fx);
    gfree(h, h->d_fy);
    gfree(h, h->d_fz);
    h->d_fx = h->d_fy = h->d_fz = nullptr;
    for (int k = 1; k <= 3; k++) {
        gfree(h, h->d_tiles[k]);
        h->d_tiles[k] = nullptr;
        h->ntiles[k] = 0;
        h->tile_smem[k] = h->tile_smem_mu[k] = 0;
    }
    for (int a = 0; a < 3; a++) h->bc[a] = kind[a];
    h->layer = any ? layer : 0;
    h->gamma_max = any ? gamma_max : 0.0;
    drop_graph(h);
    if (h->has_mu) LBEM_CUDA(launch_medium_grad_walls(h, h->stream));  // grad ln mu at the walls
    if (!any) return LBEM_OK;
    // layer factors 1 - gamma_max ((L - i)/L)^2 at distance i from the wall-adjacent site, per column / row (the
    // column table padded with 1 to the row pitch, for 16-byte loads)
    const int len[3] = {h->grid.nx, h->grid.ny, h->grid.nz}, alloc[3] = {h->grid.pitch, h->grid.ny, h->grid.nz};
    float **dst[3] = {&h->d_fx, &h->d_fy, &h->d_fz};
    for (int a = 0; a < h->dim; a++) {
        if (!kind[a] || layer == 0) continue;
        std::vector<float> f(alloc[a], 1.f);
        for (int v = 0; v < len[a]; v++) {
            const int i = std::min(v, len[a] - 1 - v);
            const double r = (double)(layer - i) / layer;
            f[v] = i < layer ? (float)(1.0 - gamma_max * r * r) : 1.f;
        }
        LBEM_CUDA(gmalloc(h, (void **)dst[a], sizeof(float) * alloc[a], "layer factors"));
        LBEM_CUDA(cudaMemcpy(*dst[a], f.data(), sizeof(float) * alloc[a], cudaMemcpyHostToDevice));
    }
    if (h->dim == 2 && !h->edge_stream) {  // the edge pass's stream and events (kept for the handle's life)
        LBEM_CUDA(cudaStreamCreateWithFlags(&h->edge_stream, cudaStreamNonBlocking));
        LBEM_CUDA(cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming));
        LBEM_CUDA(cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming));
    }
    for (int k = 1; k <= 3 && h->dim == 2; k++) {  // 2D: the edge kernel's tiles (the 3D kernel applies walls)
        const std::vector<EdgeTile> t = edge_tiles(h->grid, h->bc, h->layer, k);
        h->ntiles[k] = (int)t.size();
        h->tile_smem[k] = edge_smem_bytes(k, t, false);
        h->tile_smem_mu[k] = edge_smem_bytes(k, t, true);
        LBEM_CUDA(gmalloc(h, (void **)&h->d_tiles[k], sizeof(EdgeTile) * std::max<size_t>(t.size(), 1), "edge tiles"));
        LBEM_CUDA(cudaMemcpy(h->d_tiles[k], t.data(), sizeof(EdgeTile) * t.size(), cudaMemcpyHostToDevice));
    }
    LBEM_CUDA(cudaStreamSynchronize(h->stream));
    return LBEM_OK;
}

lbem_status lbem_set_dispersion(lbem_t *h, const float *wp2, const float *wr2, const float *gamma) {
    if (!h) return fail(LBEM_ERR_ARG, "null handle");
    if (!wp2) {  // back to a non-dispersive medium
        LBEM_CUDA(cudaStreamSynchronize(h->stream));
        for (float **p : {&h->d_wp2, &h->d_wr2, &h->d_gam, &h->d_J, &h->d_P, &h->d_P2, &h->d_pc, &h->d_pb, &h->d_pa}) {
            gfree(h, *p);
            *p = nullptr;
        }
        h->disp = false;
        drop_graph(h);
        return LBEM_OK;
    }
    if (h->dim != 2 || h->storage != LBEM_F32)
        return fail(LBEM_ERR_ARG, "lbem_set_dispersion: 2D grids with LBEM_F32 storage only");
    if (!h->has_medium) return fail(LBEM_ERR_STATE, "lbem_set_dispersion: set a medium first");
    if (h->adj) return fail(LBEM_ERR_STATE, "lbem_set_dispersion: a recorded adjoint run exists (non-dispersive only)");
    const size_t n = (size_t)h->nsite;
    const float *dp, *dr, *dg;
    lbem_status st = device_input(h, wp2, n, 0, &dp);
    if (st != LBEM_OK) return st;
    if ((st = device_input(h, wr2, n, n, &dr)) != LBEM_OK) return st;
    if ((st = device_input(h, gamma, n, 2 * n, &dg)) != LBEM_OK) return st;
    LBEM_CUDA(cudaMemsetAsync(h->d_counter, 0, sizeof(unsigned), h->stream));
    LBEM_CUDA(launch_disp_check(h, nullptr, nullptr, h->aniso_fsum(), 1.0, dp, dr, dg, false, h->d_counter,
                                h->stream));
    unsigned bad = 0;
    LBEM_CUDA(cudaMemcpyAsync(&bad, h->d_counter, sizeof(unsigned), cudaMemcpyDeviceToHost, h->stream));
    LBEM_CUDA(cudaStreamSynchronize(h->stream));
    if (bad)
        return fail(LBEM_ERR_MEDIUM, "lbem_set_dispersion: " + std::to_string(bad) +
                                         " sites with a parameter not finite and >= 0, or wp^2 + wr^2 > 4 w0");
    const size_t pl = (size_t)h->grid.plane;  // stored as planes with the grid's pitch (padding zero)
    if (!h->d_wp2) {
        for (float **p : {&h->d_wp2, &h->d_wr2, &h->d_gam, &h->d_J, &h->d_P, &h->d_P2, &h->d_pc, &h->d_pb, &h->d_pa})
            LBEM_CUDA(gmalloc(h, (void **)p, sizeof(float) * pl, "dispersive pole"));
    }
    const float *src[3] = {dp, dr, dg};
    float *dst[3] = {h->d_wp2, h->d_wr2, h->d_gam};
    for (int k = 0; k < 3; k++) LBEM_CUDA(launch_to_plane(h, src[k], dst[k], h->stream));
    LBEM_CUDA(launch_pole_coefficients(h, h->stream));
    for (float *p : {h->d_J, h->d_P, h->d_P2}) LBEM_CUDA(cudaMemsetAsync(p, 0, sizeof(float) * pl, h->stream));
    LBEM_CUDA(cudaStreamSynchronize(h->stream));
    h->disp = true;
    drop_graph(h);
    return LBEM_OK;
}

lbem_status lbem_get_boundaries(const lbem_t *h, int kind[3], int *layer, double *gamma_max) {
    if (!h) return fail(LBEM_ERR_ARG, "null handle");
    for (int a = 0; kind && a < 3; a++) kind[a] = h->bc[a];
    if (layer) *layer = h->layer;
    if (gamma_max) *gamma_max = h->gamma_max;
    return LBEM_OK;
}

lbem_status lbem_time(const lbem_t *h, long long *t) {
    if (!h || !t) return fail(LBEM_ERR_ARG, "null argument");
    *t = h->t;
    return LBEM_OK;
}

lbem_status lbem_fields(lbem_t *h, float *E, float *B) {
    if (!h) return fail(LBEM_ERR_ARG, "null handle");
    if (!h->has_medium) return fail(LBEM_ERR_STATE, "lbem_fields: set a medium first");
    if (!E && !B) return LBEM_OK;
    const size_t n3 = 3 * (size_t)h->nsite;
    const bool eh = E && !is_device_ptr(E), bh = B && !is_device_ptr(B);
    if (eh || bh) {
        lbem_status st = ensure_stage(h, 2 * n3);
        if (st != LBEM_OK) return st;
    }
    float *dE = eh ? h->d_stage : E;
    float *dB = bh ? h->d_stage + n3 : B;
    cudaError_t e = h->dim == 2 ? launch_fields_2d(h, dE, dB, h->stream) : launch_fields_3d(h, dE, dB, h->stream);
    LBEM_CUDA(e);
    if (eh) LBEM_CUDA(cudaMemcpyAsync(E, dE, n3 * sizeof(float), cudaMemcpyDeviceToHost, h->stream));
    if (bh) LBEM_CUDA(cudaMemcpyAsync(B, dB, n3 * sizeof(float), cudaMemcpyDeviceToHost, h->stream));
    if (eh || bh) LBEM_CUDA(cudaStreamSynchronize(h->stream));
    return LBEM_OK;
}

lbem_status lbem_energy_flux(lbem_t *h, float *u, float *P) {
    if (!h) return fail(LBEM_ERR_ARG, "null handle");
    if (!h->has_medium) return fail(LBEM_ERR_STATE, "lbem_energy_flux: set a medium first");
    if (!u && !P) return LBEM_OK;
    const size_t n = (size_t)h->nsite, n3 = 3 * n;
    const bool uh = u && !is_device_ptr(u), ph = P && !is_device_ptr(P);
    // staging: E, B (6n floats), then host-output copies of u (n) and P (3n)
    lbem_status st = ensure_stage(h, 2 * n3 + (uh ? n : 0) + (ph ? n3 : 0));
    if (st != LBEM_OK) return st;
    float *E = h->d_stage, *B = h->d_stage + n3;
    float *du = uh ? h->d_stage + 2 * n3 : u;
    float *dP = ph ? h->d_stage + 2 * n3 + (uh ? n : 0) : P;
    cudaError_t e = h->dim == 2 ? launch_fields_2d(h, E, B, h->stream) : launch_fields_3d(h, E, B, h->stream);
    LBEM_CUDA(e);
    LBEM_CUDA(launch_energy_flux(h, E, B, du, dP, h->stream));
    if (uh) LBEM_CUDA(cudaMemcpyAsync(u, du, n * sizeof(float), cudaMemcpyDeviceToHost, h->stream));
    if (ph) LBEM_CUDA(cudaMemcpyAsync(P, dP, n3 * sizeof(float), cudaMemcpyDeviceToHost, h->stream));
    if (uh || ph) LBEM_CUDA(cudaStreamSynchronize(h->stream));
    return LBEM_OK;
}

lbem_status lbem_traces(lbem_t *h, float *out, int *nrecorded) {
    if (!h) return fail(LBEM_ERR_ARG, "null handle");
    const int n = (int)std::min<long long>(h->t, h->cap);
    if (nrecorded) *nrecorded = n;
    if (!out || n == 0 || h->nrec == 0) return LBEM_OK;
    LBEM_CUDA(cudaMemcpy2DAsync(out, (size_t)n * sizeof(float), h->d_traces, (size_t)h->cap * sizeof(float),
                                (size_t)n * sizeof(float), h->nrec, cudaMemcpyDefault, h->stream));
    if (!is_device_ptr(out)) LBEM_CUDA(cudaStreamSynchronize(h->stream));
    return LBEM_OK;
}

lbem_status lbem_diagnostics(lbem_t *h, double out[3]) {
    if (!h || !out) return fail(LBEM_ERR_ARG, "null argument");
    if (!h->has_medium) return fail(LBEM_ERR_STATE, "lbem_diagnostics: set a medium first");
    cudaError_t e = h->dim == 2 ? launch_diag_2d(h, h->d_partials, h->n_partials, h->stream)
                                : launch_diag_3d(h, h->d_partials, h->n_partials, h->stream);
    LBEM_CUDA(e);
    LBEM_CUDA(launch_reduce_partials(h->d_partials, h->n_partials, h->d_diag, h->stream));
    LBEM_CUDA(cudaMemcpyAsync(out, h->d_diag, 3 * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    LBEM_CUDA(cudaStreamSynchronize(h->stream));
    out[2] = sqrt(out[2]);  // the kernels sum (div B)^2
    for (int k = 0; k < 3; k++)
        if (!isfinite(out[k])) return fail(LBEM_ERR_UNSTABLE, "lbem_diagnostics: non-finite state");
    return LBEM_OK;
}

lbem_status lbem_save_state(lbem_t *h, void *dst) {
    if (!h || !dst) return fail(LBEM_ERR_ARG, "null argument");
    const PopBuf &p = h->buf[h->cur];
    const size_t db = (size_t)h->npop * p.plane * elem_bytes(h->storage);
    LBEM_CUDA(cudaMemcpyAsync(dst, p.data, db, cudaMemcpyDefault, h->stream));
    if (p.ex) LBEM_CUDA(cudaMemcpyAsync((char *)dst + db, p.ex, (size_t)h->npop * p.explane, cudaMemcpyDefault, h->stream));
    if (h->disp) {  // then the pole's J and P planes
        const size_t pb = sizeof(float) * (size_t)h->grid.plane;
        LBEM_CUDA(cudaMemcpyAsync((char *)dst + db, h->d_J, pb, cudaMemcpyDefault, h->stream));
        LBEM_CUDA(cudaMemcpyAsync((char *)dst + db + pb, h->pole_P(h->cur), pb, cudaMemcpyDefault, h->stream));
    }
    if (!is_device_ptr(dst)) LBEM_CUDA(cudaStreamSynchronize(h->stream));
    return LBEM_OK;
}

lbem_status lbem_load_state(lbem_t *h, const void *src, long long t_at_save) {
    if (!h || !src || t_at_save < 0) return fail(LBEM_ERR_ARG, "lbem_load_state: bad argument");
    const PopBuf &p = h->buf[h->cur];
    const size_t db = (size_t)h->npop * p.plane * elem_bytes(h->storage);
    LBEM_CUDA(cudaMemcpyAsync(p.data, src, db, cudaMemcpyDefault, h->stream));
    if (p.ex)
        LBEM_CUDA(cudaMemcpyAsync(p.ex, (const char *)src + db, (size_t)h->npop * p.explane, cudaMemcpyDefault, h->stream));
    if (h->disp) {
        const size_t pb = sizeof(float) * (size_t)h->grid.plane;
        LBEM_CUDA(cudaMemcpyAsync(h->d_J, (const char *)src + db, pb, cudaMemcpyDefault, h->stream));
        LBEM_CUDA(cudaMemcpyAsync(h->pole_P(h->cur), (const char *)src + db + pb, pb, cudaMemcpyDefault, h->stream));
    }
    if (!is_device_ptr(src)) LBEM_CUDA(cudaStreamSynchronize(h->stream));
    h->t = t_at_save;
    drop_graph(h);
    return LBEM_OK;
}

lbem_status lbem_rows(lbem_t *h, int plane, int row0, int nrows, float *buf, int to_state) {
    if (!h || !buf) return fail(LBEM_ERR_ARG, "null argument");
    if (h->storage != LBEM_F32) return fail(LBEM_ERR_ARG, "lbem_rows: LBEM_F32 storage only");
    if (plane < 0 || plane >= h->npop || nrows < 0 || row0 < 0 || row0 + nrows > h->grid.nrows)
        return fail(LBEM_ERR_ARG, "lbem_rows: plane or rows out of range");
    if (nrows == 0) return LBEM_OK;
    const PopBuf &p = h->buf[h->cur];
    float *base = static_cast<float *>(p.data) + (long long)plane * p.plane + (long long)row0 * p.pitch;
    const size_t w = sizeof(float) * (size_t)h->grid.nx, pitch = sizeof(float) * (size_t)p.pitch;
    if (to_state) LBEM_CUDA(cudaMemcpy2DAsync(base, pitch, buf, w, w, nrows, cudaMemcpyDefault, h->stream));
    else LBEM_CUDA(cudaMemcpy2DAsync(buf, w, base, pitch, w, nrows, cudaMemcpyDefault, h->stream));
    if (!is_device_ptr(buf)) LBEM_CUDA(cudaStreamSynchronize(h->stream));
    return LBEM_OK;  // (a cached graph depends on the buffers and parameters, not on their contents)
}

static lbem_status halo_rows(lbem_t *h, int halo, float *up, float *down, int to_state, const char *who) {
    const std::string name(who);
    if (!h) return fail(LBEM_ERR_ARG, "null handle");
    if (h->dim != 2 || h->storage != LBEM_F32) return fail(LBEM_ERR_ARG, name + ": 2D LBEM_F32 handles only");
    if (halo != 1 && halo != 2) return fail(LBEM_ERR_ARG, name + ": halo must be 1 or 2");
    if (h->grid.ny < 3 * halo) return fail(LBEM_ERR_ARG, name + ": a slab needs at least 3 * halo rows");
    for (float *b : {up, down})
        if (b && !is_device_ptr(b)) return fail(LBEM_ERR_ARG, name + ": buffers must be device memory");
    const PopBuf &p = h->buf[h->cur];
    float *state = static_cast<float *>(p.data);
    const int nx = h->grid.nx;
    for (int k = 0; k < 2; k++) {
        float *b = k ? down : up;
        if (!b) continue;
        const HaloRows spec = halo_spec(halo, h->grid.ny, k == 0, !to_state);
        const dim3 grid((unsigned)std::min((nx + 255) / 256, 64), (unsigned)spec.n);
        halo_rows_kernel<<<grid, 256, 0, h->stream>>>(state, p.plane, p.pitch, nx, spec, b, to_state);
        LBEM_CUDA(cudaGetLastError());
    }
    return LBEM_OK;
}

lbem_status lbem_halo_out(lbem_t *h, int halo, float *up, float *down) {
    return halo_rows(h, halo, up, down, 0, "lbem_halo_out");
}

lbem_status lbem_halo_in(lbem_t *h, int halo, const float *from_below, const float *from_above) {
    // the rows from below fill the lower ghost rows, those from above the upper ones
    return halo_rows(h, halo, const_cast<float *>(from_above), const_cast<float *>(from_below), 1, "lbem_halo_in");
}

lbem_status lbem_check_guards(lbem_t *h) {
    if (!h) return fail(LBEM_ERR_ARG, "null handle");
    LBEM_CUDA(cudaStreamSynchronize(h->stream));
    if (tb2_take_timeouts())
        return fail(LBEM_ERR_TIMEOUT, "lbem_check_guards: a tile load of the two-step kernel did not complete");
    std::vector<unsigned char> buf(2 * GUARD);
    for (const auto &g : h->guarded) {
        const char *u = static_cast<const char *>(g.user);
        LBEM_CUDA(cudaMemcpy(buf.data(), u - GUARD, GUARD, cudaMemcpyDeviceToHost));
        LBEM_CUDA(cudaMemcpy(buf.data() + GUARD, u + g.bytes, GUARD, cudaMemcpyDeviceToHost));
        for (size_t i = 0; i < buf.size(); i++)
            if (buf[i] != GUARD_BYTE)
                return fail(LBEM_ERR_STATE, std::string("lbem_check_guards: guard band ") +
                                                (i < GUARD ? "before" : "after") + " array '" + g.name +
                                                "' overwritten");
    }
    return LBEM_OK;
}

lbem_status lbem_set_variant(lbem_t *h, int variant) {
    if (!h) return fail(LBEM_ERR_ARG, "null handle");
    const int nv = h->dim == 2 ? nvariants_2d() : nvariants_3d();
    if (variant < 0 || variant >= nv) return fail(LBEM_ERR_ARG, "lbem_set_variant: out of range");
    h->variant = variant;
    drop_graph(h);
    return LBEM_OK;
}

lbem_status lbem_get_variant(const lbem_t *h, int *variant, int *nvariants) {
    if (!h) return fail(LBEM_ERR_ARG, "null handle");
    if (variant) *variant = h->variant;
    if (nvariants) *nvariants = h->dim == 2 ? nvariants_2d() : nvariants_3d();
    return LBEM_OK;
}

lbem_status lbem_autotune(lbem_t *h, int trial_steps, int *best) {
    if (!h) return fail(LBEM_ERR_ARG, "null handle");
    if (!h->has_medium) return fail(LBEM_ERR_STATE, "lbem_autotune: set a medium first");
    if (trial_steps < 1) return fail(LBEM_ERR_ARG, "lbem_autotune: trial_steps >= 1");
    if (h->general()) {  // a dispersive or anisotropic handle has one kernel
        if (best) *best = h->variant;
        return LBEM_OK;
    }
    const int nv = h->dim == 2 ? nvariants_2d() : nvariants_3d();
    size_t bytes = 0;
    lbem_info(h, nullptr, &bytes);
    void *save = nullptr;
    if (cudaMalloc(&save, bytes) != cudaSuccess) {
        cudaGetLastError();
        return fail(LBEM_ERR_NOMEM, "lbem_autotune: no room to save the state");
    }
    const int cur0 = h->cur;
    const long long t0 = h->t;
    lbem_status st = lbem_save_state(h, save);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best_ms = 1e30f;
    int best_v = h->variant;
    for (int v = 0; v < nv && st == LBEM_OK; v++) {
        int cur = cur0;
        for (int rep = 0; rep < 2 && st == LBEM_OK; rep++) {  // first pass warms up
            cudaEventRecord(e0, h->stream);
            for (int n = 0; n < trial_steps; n++) {
                StepArgs a = step_args(h, cur);
                a.evt.rowptr = nullptr;  // no trace writes while timing
                cudaError_t e = launch_step(h, a, v);
                if (e != cudaSuccess) {
                    st = cuda_fail(e, "lbem_autotune");
                    break;
                }
                cur ^= 1;
            }
            cudaEventRecord(e1, h->stream);
        }
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best_ms) {
            best_ms = ms;
            best_v = v;
        }
    }
    // two and three steps per launch (where enabled and applicable): time every tile shape; keep the fastest
    // per step, single steps included
    float best_per_step = best_ms / trial_steps;
    int best_shape = h->tb_shape, best_tblock = 1;
    const int max_k = h->tblock;
    for (int k = 2; k <= max_k && st == LBEM_OK; k++) {
        if (!multi_step_base(h) || (k == 3 && (h->storage != LBEM_F32 || h->has_mu))) continue;
        const int nl = trial_steps / k > 0 ? trial_steps / k : 1;
        const int nsh = k == 3 ? tb3_nshapes() : two_step_nshapes(h);
        for (int shape = 0; shape < nsh && st == LBEM_OK; shape++) {
            int cur = cur0;
            for (int rep = 0; rep < 2 && st == LBEM_OK; rep++) {
                cudaEventRecord(e0, h->stream);
                for (int n = 0; n < nl; n++) {
                    StepArgs a = step_args(h, cur);
                    a.evt.rowptr = nullptr;
                    cudaError_t e = k == 3 ? launch_step_2d_tb3(a, shape, h->stream)
                                           : launch_step_2d_tb2(a, h->storage, shape, h->stream);
                    if (e != cudaSuccess) {
                        st = cuda_fail(e, "lbem_autotune");
                        break;
                    }
                    cur ^= 1;
                }
                cudaEventRecord(e1, h->stream);
            }
            cudaEventSynchronize(e1);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (ms / (k * nl) < best_per_step) {
                best_per_step = ms / (k * nl);
                best_shape = shape;
                best_tblock = k;
            }
        }
    }
    if (best_tblock == 1) best_shape = 0;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    h->cur = cur0;
    if (st == LBEM_OK) st = lbem_load_state(h, save, t0);
    cudaStreamSynchronize(h->stream);
    cudaFree(save);
    if (st != LBEM_OK) return st;
    h->variant = best_v;
    h->tb_shape = best_shape;
    h->tb_shape_set = true;
    h->tblock = best_tblock;
    drop_graph(h);
    if (best) *best = best_v;
    return LBEM_OK;
}

lbem_status lbem_get_temporal_blocking(const lbem_t *h, int *steps_per_pass, int *tile_shape, int *nshapes) {
    if (!h) return fail(LBEM_ERR_ARG, "null handle");
    if (steps_per_pass) *steps_per_pass = steps_per_launch(h);
    if (tile_shape) *tile_shape = steps_per_launch(h) == 2 ? two_step_shape(h) : h->tb_shape;
    if (nshapes) *nshapes = h->tblock == 3 ? tb3_nshapes() : two_step_nshapes(h);
    return LBEM_OK;
}

}  // extern "C"
