// runtime.cu -- the C ABI of include/lbm.h: handle, device memory through an
// allocator hook, the step as a CUDA graph per step parity, the device status
// word, field export / import, history, checkpoint and kernel timing.
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>
#include <cmath>
#include <algorithm>
#include <climits>

#include "../../include/lbm.h"
#include "lbm_internal.cuh"

using lbm::BodyProps;
using lbm::BodyState;
using lbm::DriveTerm;
using lbm::Spring;

namespace {
constexpr int CHUNK_STEPS = 16;     // steps per chunk graph (even)
const char SAVE_MAGIC[8] = {'L', 'B', 'M', '3', 'S', 'A', 'V', '1'};
}  // namespace

struct lbm_s {
    // configuration (host)
    int nx = 0, ny = 0, nz = 0, bc = 0, precision = 1, options = 0;
    double tau = 1.0, g[3] = {0, 0, 0};
    long long C = 0;
    std::vector<BodyProps> props;
    std::vector<BodyState> init_state;
    std::vector<Spring> springs;
    std::vector<DriveTerm> drives;
    int hist_cap = 0;
    int tune_vec = 0, tune_minb = 0;
    // the next step needs the body preparation (geometry records of states
    // the rigid-body step did not make; set when the host writes a state)
    bool need_prep = true;
    int expire_waits = 0;               // lbm_debug_set knobs
    int adjoint_sets = 0;
    int no_pdl = 1;         // LBM_DEBUG_NO_PDL: step graphs without programmatic dependent launch
    long long list_cap_limit = 0;
    // asynchronous reads (lbm_get_bodies_async): a ring of completion events
    // and pinned status words, one per read ticket modulo READS
    static constexpr int READS = 64;
    cudaEvent_t rd_ev[READS] = {};
    int *rd_status = nullptr;
    long long rd_seq = 0;
    // the reads run on a stream of their own beside the following step; a
    // step that overwrites a body buffer with a read pending waits for it
    cudaStream_t rd_stream = nullptr;
    cudaEvent_t rd_after = nullptr;
    int rd_pending[2] = {-1, -1};           // ring slot of the last read of body buffer p, or -1
    double *avg_sum = nullptr;          // [3][C] running velocity sum (lbm_average_*)
    long long *avg_count = nullptr;     // steps added to it (device)
    unsigned graph_gen = 0;             // bumped whenever the step graphs are rebuilt with other kernels
    std::vector<int> drive_slot;        // creation index of each device drive term (grouped by body)
    // device
    bool ready = false, graphs_ready = false;
    int device = 0;
    cudaStream_t stream = nullptr, cap = nullptr, side = nullptr;
    cudaEvent_t fork_ev = nullptr, join_ev = nullptr;
    // a third branch of the step graphs: the link lists and loads beside the
    // boundary kernel (a small lattice's bulk kernel is shorter than both)
    cudaStream_t side2 = nullptr;
    cudaEvent_t join2_ev = nullptr;
    // overlapped steps: the far bulk kernels' stream, and by step parity the
    // events "far bulk of step n done" and "near cells of step n done"
    cudaStream_t far = nullptr;
    cudaEvent_t far_ev[2] = {nullptr, nullptr}, near_ev[2] = {nullptr, nullptr};
    bool tiles_stale = false;           // the host set a body state: redo the next step's near tiles
    lbm_alloc_fn afn = nullptr;
    lbm_free_fn ffn = nullptr;
    void *actx = nullptr;
    std::vector<void *> allocs;
    lbm::Device dv{};
    void *pop[2] = {nullptr, nullptr};
    uint8_t *flags[2] = {nullptr, nullptr}, *bid[2] = {nullptr, nullptr};
    BodyState *bodies[2] = {nullptr, nullptr};
    long long steps = 0;
    cudaGraphExec_t single[2] = {nullptr, nullptr};
    cudaGraphExec_t chunk = nullptr;
    // reverse sweep: the recording of the last lbm_adjoint_record
    struct Tape {
        bool recorded = false;
        int n = 0, seg = 0, nseg = 0;
        long long n0 = 0;
        lbm::TapeCtl *ctl = nullptr;        // device switch read by the rigid-body step
        lbm::TapeCtl ctl_host{};
        double *state = nullptr;            // [n + 2][nb][13]: states n0 - 1 ... n0 + n
        double *force = nullptr;            // [n][nb][6]
        void *ckpt_pop = nullptr;           // [nseg][19][C]: populations entering each segment
        uint8_t *ckpt_flags = nullptr, *ckpt_bid = nullptr;   // [nseg][C]: epoch before each segment
        std::vector<void *> allocs;
    } tape;
    std::string err;
};

namespace {

int fail(lbm_t *h, int code, const char *fmt, ...) {
    if (h) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        h->err = buf;
    }
    return code;
}

int cuda_fail(lbm_t *h, cudaError_t e, const char *what) {
    return fail(h, LBM_E_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define CK(call)                                              \
    do {                                                      \
        cudaError_t e_ = (call);                              \
        if (e_ != cudaSuccess) return cuda_fail(h, e_, #call); \
    } while (0)

size_t pop_bytes(int precision) { return precision == 0 ? 8 : (precision == 1 ? 4 : 2); }

void *dalloc(lbm_t *h, size_t bytes) {
    if (bytes == 0) bytes = 256;
    void *p = nullptr;
    if (h->afn) {
        p = h->afn(bytes, h->actx);
    } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
        p = nullptr;
    }
    return p;
}

void dfree(lbm_t *h, void *p) {
    if (!p) return;
    if (h->afn) {
        if (h->ffn) h->ffn(p, h->actx);
    } else {
        cudaFree(p);
    }
}

template <typename T>
int alloc_into(lbm_t *h, T **out, size_t bytes) {
    void *p = dalloc(h, bytes);
    if (!p) return fail(h, LBM_E_OOM, "device allocation of %zu bytes failed", bytes);
    h->allocs.push_back(p);
    *out = static_cast<T *>(p);
    return LBM_OK;
}

bool fluid(const lbm_t *h) { return !(h->options & LBM_OPT_NO_FLUID); }
int nb(const lbm_t *h) { return (int)h->props.size(); }

// the step pointers of parity p; `overlap`: the bulk kernel leaves the near
// tiles to the near kernel and the step index comes from the near-tile kernel
lbm::StepPtrs step_ptrs(lbm_t *h, int p, bool overlap = false) {
    const int q = p ^ 1;
    lbm::StepPtrs sp{};
    overlap = overlap && h->dv.overlap;
    sp.far_skip = overlap ? h->dv.near_mask[p] : nullptr;
    sp.tstep = overlap ? h->dv.tstep + p : h->dv.t_dev;
    sp.src = h->pop[q];
    sp.dst = h->pop[p];
    sp.flags_prev = h->flags[q];
    sp.bid_prev = h->bid[q];
    sp.flags_cur = h->flags[p];
    sp.bid_cur = h->bid[p];
    sp.body_prev = h->bodies[q];
    sp.body_cur = h->bodies[p];
    sp.body_next = h->bodies[q];
    sp.parity = p;
    return sp;
}

// the kernels of one step of parity p, in Algorithm 2's order; `ev`
// (optional) brackets each kernel slot with a pair of events.  With `fork`
// the boundary-cell kernel, then the link lists and the drive and spring
// loads, run on a second stream concurrently with the bulk kernel (they
// touch no data the bulk kernel reads or writes) and join before the force
// sums.
void enqueue_overlapped(lbm_t *h, int p, cudaStream_t s, bool first);

void enqueue_step(lbm_t *h, int p, cudaStream_t s, cudaEvent_t *ev = nullptr, bool *ran = nullptr,
                  bool fork = false, bool prep = true) {
    const lbm::StepPtrs sp = step_ptrs(h, p);
    const bool bodies = nb(h) > 0, fl = fluid(h);
    auto run = [&](int slot, cudaStream_t st, auto &&fn) {
        if (ev) cudaEventRecord(ev[2 * slot], st);
        fn();
        if (ev) cudaEventRecord(ev[2 * slot + 1], st);
        if (ran) ran[slot] = true;
    };
    if (bodies && fl) run(LBM_KERNEL_REMAP, s, [&] { lbm::launch_remap(h->dv, sp, 0, s, prep); });
    const bool boundary = fl && lbm::needs_boundary_fix(h->dv);
    const bool forked = boundary && fork;
    if (forked) {
        cudaEventRecord(h->fork_ev, s);
        cudaStreamWaitEvent(h->side, h->fork_ev, 0);
        lbm::launch_boundary_fix(h->dv, sp, h->side);
        cudaEventRecord(h->join_ev, h->side);
        if (bodies) {
            cudaStreamWaitEvent(h->side2, h->fork_ev, 0);
            lbm::launch_links(h->dv, sp, h->side2);
            cudaEventRecord(h->join2_ev, h->side2);
        }
    }
    if (fl) run(LBM_KERNEL_STREAM_COLLIDE, s, [&] {
        // the bulk kernel waits for the remap in full: launched before the
        // remap ends, its blocks would hold every SM ahead of the boundary
        // branch, which is launched when the remap ends
        lbm::Device dvb = h->dv;
        dvb.pdl = 0;
        lbm::launch_stream_collide(dvb, sp, s);
    });
    if (boundary && !forked) run(LBM_KERNEL_BOUNDARY, s, [&] { lbm::launch_boundary_fix(h->dv, sp, s); });
    if (bodies && fl && !forked) run(LBM_KERNEL_LINKS, s, [&] { lbm::launch_links(h->dv, sp, s); });
    if (forked) {
        cudaStreamWaitEvent(s, h->join_ev, 0);
        if (bodies) cudaStreamWaitEvent(s, h->join2_ev, 0);
    }
    if (bodies && fl) {
        // momentum exchange; the last block of each body runs its rigid-body step
        run(LBM_KERNEL_FORCE, s, [&] { lbm::launch_force(h->dv, sp, s); });
    } else if (bodies) {
        run(LBM_KERNEL_INTEGRATE, s, [&] { lbm::launch_integrate(h->dv, sp, 0, s); });
    } else if (fl) {
        lbm::launch_tick(h->dv, sp, s);             // the step counter of a lattice without bodies
    }
    // the running velocity average reads the populations this step wrote
    if (fl && h->dv.avg_u) lbm::launch_average(h->dv, sp, s);
}

// One overlapped step n of parity p (lattices with bodies and fluid).  Two
// streams: the chain s (remap, links, loads, boundary and near cells, the
// next step's near tiles, force + rigid-body step) and the far stream (the
// bulk kernel outside the near tiles).  far(n) waits for the near cells of
// step n-1 (its sources; the chain of step n-1 also made step n's near
// tiles); the near and boundary cells of step n wait for far(n-1), which
// reads the buffer they write.  So far(n) runs beside force(n-1), remap(n)
// and everything else of step n.  `first`: the first step of a capture
// (its predecessors completed before the graph started).
void enqueue_overlapped(lbm_t *h, int p, cudaStream_t s, bool first) {
    const lbm::StepPtrs sp = step_ptrs(h, p, true);
    const int q = p ^ 1;
    // far stream: wait for step n-1's near cells, then the far bulk kernel
    if (first) {
        cudaEventRecord(h->fork_ev, s);
        cudaStreamWaitEvent(h->far, h->fork_ev, 0);
    } else {
        cudaStreamWaitEvent(h->far, h->near_ev[q], 0);
    }
    lbm::launch_stream_collide(h->dv, sp, h->far);
    cudaEventRecord(h->far_ev[p], h->far);
    // the chain
    lbm::launch_remap(h->dv, sp, 0, s);
    lbm::launch_links(h->dv, sp, s);
    if (!first) cudaStreamWaitEvent(s, h->far_ev[q], 0);
    lbm::launch_boundary_fix(h->dv, sp, s);
    lbm::launch_near_bulk(h->dv, sp, s);
    lbm::launch_near_tiles(h->dv, sp.body_cur, q, 1, s);        // step n+1's, from state n
    cudaEventRecord(h->near_ev[p], s);
    lbm::launch_force(h->dv, sp, s);
    if (h->dv.avg_u) {
        cudaStreamWaitEvent(s, h->far_ev[p], 0);
        lbm::launch_average(h->dv, sp, s);
    }
}

// the step graphs bake in the kernels and their arguments: drop them so that
// the next step rebuilds them
void drop_graphs(lbm_t *h) {
    for (int p = 0; p < 2; ++p)
        if (h->single[p]) { cudaGraphExecDestroy(h->single[p]); h->single[p] = nullptr; }
    if (h->chunk) { cudaGraphExecDestroy(h->chunk); h->chunk = nullptr; }
    h->graphs_ready = false;
    ++h->graph_gen;
}

bool overlapped(const lbm_t *h) {
    return fluid(h) && nb(h) > 0 && (h->options & LBM_OPT_OVERLAP);
}

int kernels_per_step(const lbm_t *h) {
    const bool bodies = nb(h) > 0, fl = fluid(h);
    const bool walls = (h->bc & 7) != 7;
    int n = 0;
    if (bodies && fl) n += overlapped(h) ? 2 : 1;           // (body preparation,) remap
    if (fl) n += 1;                                         // bulk stream-collide
    if (fl) n += (bodies ? 1 : 0) + (walls ? 1 : 0);        // boundary cells
    if (bodies && fl) n += 3;                               // links, drive and spring loads, force + rigid-body step
    if (bodies && !fl) n += 1;                              // rigid-body step alone
    if (!bodies && fl) n += 1;                              // step counter
    if (fl && h->dv.avg_u) n += 1;                          // running velocity average
    if (overlapped(h)) n += 2;                              // near cells, next step's near tiles
    return n;
}

// flags of the epoch before the first step: the mapping of state 0
int init_flags(lbm_t *h) {
    lbm::launch_init_flags(h->dv, h->flags[0], h->flags[1], h->bid[0], h->bid[1], h->stream);
    if (nb(h) > 0 && fluid(h)) {
        lbm::StepPtrs sp = step_ptrs(h, 1);
        sp.body_cur = h->bodies[0];
        lbm::launch_remap(h->dv, sp, 1, h->stream);
    }
    // the first step's near tiles
    if (h->dv.overlap) lbm::launch_near_tiles(h->dv, h->bodies[0], 0, 0, h->stream);
    h->tiles_stale = false;
    CK(cudaGetLastError());
    return LBM_OK;
}

// the next step's near tiles from the current body states, after the host
// set a state or steps ran without the overlapped graphs
int refresh_tiles(lbm_t *h) {
    if (!h->tiles_stale) return LBM_OK;
    if (h->dv.overlap) {
        const int p = (int)(h->steps & 1);
        lbm::launch_near_tiles(h->dv, h->bodies[p], p, 0, h->stream);
        CK(cudaGetLastError());
    }
    h->tiles_stale = false;
    return LBM_OK;
}

int upload_bodies(lbm_t *h) {
    h->need_prep = true;
    const size_t bs = sizeof(BodyState) * nb(h);
    if (!bs) return LBM_OK;
    CK(cudaMemcpyAsync(h->bodies[0], h->init_state.data(), bs, cudaMemcpyHostToDevice, h->stream));
    CK(cudaMemcpyAsync(h->bodies[1], h->init_state.data(), bs, cudaMemcpyHostToDevice, h->stream));
    return LBM_OK;
}

int ensure_device(lbm_t *h) {
    if (h->ready) return LBM_OK;
    CK(cudaGetDevice(&h->device));
    lbm::prepare_bulk_variants();
    int rc;
    const size_t es = pop_bytes(h->precision);
    const long long C = h->C;
    const int B = nb(h);
    int emax = 0;
    for (const auto &p : h->props) emax = std::max(emax, p.E);
    lbm::Device &dv = h->dv;
    dv.dom = lbm::Domain{h->nx, h->ny, h->nz, (h->bc & 1) ? 1 : 0, (h->bc & 2) ? 1 : 0, (h->bc & 4) ? 1 : 0, C,
                         1.0 / h->nx, 1.0 / h->ny, 1.0 / h->nz};
    dv.precision = h->precision;
    dv.nb = B;
    dv.ns = (int)h->springs.size();
    dv.nd = (int)h->drives.size();
    dv.tau = h->tau;
    dv.omega = 1.0 / h->tau;
    for (int i = 0; i < 3; ++i) dv.g[i] = h->g[i];
    dv.omega_f = (float)dv.omega;
    dv.guo_f = (float)(1.0 - 0.5 * dv.omega);
    for (int i = 0; i < 3; ++i) dv.g_f[i] = (float)dv.g[i];
    dv.om1_f = (float)(1.0 - dv.omega);
    {
        const double wc[3] = {1.0 / 3.0, 1.0 / 18.0, 1.0 / 36.0};
        for (int i = 0; i < 3; ++i) {
            dv.ow_f[i] = (float)(dv.omega * wc[i]);
            dv.gw_f[i] = (float)((1.0 - 0.5 * dv.omega) * wc[i]);
        }
    }
    dv.forced = (h->g[0] != 0.0 || h->g[1] != 0.0 || h->g[2] != 0.0) ? 1 : 0;
    dv.avg_force = (h->options & LBM_OPT_AVERAGE_FORCE) ? 1 : 0;
    dv.f16_scale = h->precision == LBM_PREC_F16 ? 1024.0f : 1.0f;
    dv.f16_inv_scale = 1.0f / dv.f16_scale;
    dv.remap_side = 2 * (emax + lbm::REMAP_MARGIN) + 1;
    dv.link_side = 2 * (emax + 1) + 1;
    dv.seg_cap = dv.link_side * dv.link_side * 18;
    dv.hist_cap = h->hist_cap;
    dv.vec = h->tune_vec ? h->tune_vec : lbm::default_vector_width(dv);
    dv.minb = h->tune_minb;
    dv.expire_waits = h->expire_waits;

    // per-body reciprocals and term lists (drive terms and springs keep
    // their creation order within a body)
    std::vector<BodyProps> props_h = h->props;
    std::vector<DriveTerm> drives_h;
    std::vector<int> spring_list;
    for (int b = 0; b < B; ++b) {
        BodyProps &p = props_h[b];
        p.inv_m = 1.0 / p.m;
        for (int i = 0; i < 3; ++i) p.inv_inertia[i] = 1.0 / p.inertia[i];
        p.drive_first = (int)drives_h.size();
        for (size_t k = 0; k < h->drives.size(); ++k) {
            const DriveTerm &d = h->drives[k];
            if (d.body == b) {
                DriveTerm t = d;
                t.omega = 2.0 * M_PI * d.freq;
                t.t_on = d.phase / t.omega;
                drives_h.push_back(t);
                h->drive_slot.push_back((int)k);
            }
        }
        p.drive_count = (int)drives_h.size() - p.drive_first;
        p.spring_first = (int)spring_list.size();
        for (size_t k = 0; k < h->springs.size(); ++k)
            if (h->springs[k].i == b || h->springs[k].j == b) spring_list.push_back((int)k);
        p.spring_count = (int)spring_list.size() - p.spring_first;
    }

    for (int i = 0; i < 2; ++i) {
        if ((rc = alloc_into(h, &h->pop[i], es * lbm::Q * C))) return rc;
        if ((rc = alloc_into(h, &h->flags[i], (size_t)C))) return rc;
        if ((rc = alloc_into(h, &h->bid[i], (size_t)C))) return rc;
        if ((rc = alloc_into(h, &h->bodies[i], sizeof(BodyState) * std::max(B, 1)))) return rc;
    }
    BodyProps *props; Spring *springs; DriveTerm *drives;
    if ((rc = alloc_into(h, &props, sizeof(BodyProps) * std::max(B, 1)))) return rc;
    if ((rc = alloc_into(h, &springs, sizeof(Spring) * std::max<size_t>(h->springs.size(), 1)))) return rc;
    if ((rc = alloc_into(h, &drives, sizeof(DriveTerm) * std::max<size_t>(h->drives.size(), 1)))) return rc;
    if ((rc = alloc_into(h, &dv.fh, sizeof(double) * 6 * std::max(B, 1)))) return rc;
    if ((rc = alloc_into(h, &dv.fpart, sizeof(double) * 6 * lbm::FORCE_BLOCKS * std::max(B, 1)))) return rc;
    if ((rc = alloc_into(h, &dv.fx, sizeof(long long) * 6 * std::max(B, 1)))) return rc;
    if ((rc = alloc_into(h, &dv.fi, sizeof(int) * 6 * std::max(B, 1)))) return rc;
    if ((rc = alloc_into(h, &dv.geom, sizeof(lbm::BodyGeom) * 2 * std::max(B, 1)))) return rc;
    if ((rc = alloc_into(h, &dv.gstamp, sizeof(BodyState) * 2 * std::max(B, 1)))) return rc;
    {
        // every cube cell is listed at most once per body cube, and a cell
        // lies in few cubes: the smaller of the two bounds below (the
        // remap checks the capacity and reports an overflow)
        const long long rs = dv.remap_side;
        const long long cubes = (long long)B * rs * rs * rs, two_c = 2 * C + 1024;
        const size_t cap = B > 0 && fluid(h) ? (size_t)std::min(cubes, two_c) : 1;
        dv.blist_cap = h->list_cap_limit > 0 ? std::min((long long)cap, h->list_cap_limit) : (long long)cap;
        if ((rc = alloc_into(h, &dv.blist, sizeof(uint32_t) * cap))) return rc;
        if ((rc = alloc_into(h, &dv.cand, (size_t)std::max(B, 1) * std::max(B, 1)))) return rc;
        // the boundary cells' densities for the momentum exchange (32/16-bit
        // storage; written and read only at cells the boundary kernel collides)
        const bool need_rho = B > 0 && fluid(h) && h->precision != LBM_PREC_F64;
        if ((rc = alloc_into(h, &dv.rho_near, sizeof(float) * (need_rho ? (size_t)C : 1)))) return rc;
        if ((rc = alloc_into(h, &dv.bcount, sizeof(int) * 4))) return rc;
    }
    int *slist;
    if ((rc = alloc_into(h, &slist, sizeof(int) * std::max<size_t>(spring_list.size(), 1)))) return rc;
    dv.spring_list = slist;
    if ((rc = alloc_into(h, &dv.drive_f, sizeof(double) * 3 * std::max<size_t>(h->drives.size(), 1)))) return rc;
    if ((rc = alloc_into(h, &dv.spring_f, sizeof(double) * 3 * std::max<size_t>(h->springs.size(), 1)))) return rc;
    if ((rc = alloc_into(h, &dv.blocks_done, sizeof(unsigned) * 4))) return rc;
    if ((rc = alloc_into(h, &dv.body_done, sizeof(unsigned) * std::max(B, 1)))) return rc;
    const size_t nlinks = (size_t)std::max(B, 1) * dv.link_side * dv.seg_cap;
    if ((rc = alloc_into(h, &dv.links, sizeof(lbm::Link) * (B > 0 && fluid(h) ? nlinks : 1)))) return rc;
    if ((rc = alloc_into(h, &dv.seg_count, sizeof(int) * std::max(B, 1) * dv.link_side))) return rc;
    if ((rc = alloc_into(h, &dv.status, sizeof(int) * 4))) return rc;
    dv.changed = dv.status + 2;
    if ((rc = alloc_into(h, &dv.t_dev, sizeof(long long)))) return rc;
    if ((rc = alloc_into(h, &dv.tstep, sizeof(long long) * 2))) return rc;
    dv.overlap = overlapped(h) ? 1 : 0;
    dv.near_cap = dv.overlap ? lbm::near_tile_cap(dv, emax) : 0;
    for (int i = 0; i < 2; ++i) {
        const size_t tiles = dv.overlap ? (size_t)lbm::near_tile_count(dv) : 1;
        if ((rc = alloc_into(h, &dv.near_mask[i], sizeof(unsigned) * tiles))) return rc;
        if ((rc = alloc_into(h, &dv.near_list[i], sizeof(int) * std::max(dv.near_cap, 1)))) return rc;
    }
    if ((rc = alloc_into(h, &dv.near_count, sizeof(int) * 2))) return rc;
    dv.hist = nullptr;
    if (h->hist_cap > 0 && (rc = alloc_into(h, &dv.hist, sizeof(double) * 13 * h->hist_cap * std::max(B, 1))))
        return rc;
    dv.props = props;
    dv.springs = springs;
    dv.drives = drives;
    if ((rc = alloc_into(h, &h->tape.ctl, sizeof(lbm::TapeCtl)))) return rc;
    dv.tape = h->tape.ctl;

    cudaStream_t s = h->stream;
    CK(cudaMemsetAsync(h->pop[0], 0, es * lbm::Q * C, s));   // deviation 0: fluid at rest
    CK(cudaMemsetAsync(h->pop[1], 0, es * lbm::Q * C, s));
    CK(cudaMemsetAsync(dv.fh, 0, sizeof(double) * 6 * std::max(B, 1), s));
    CK(cudaMemsetAsync(dv.fpart, 0, sizeof(double) * 6 * lbm::FORCE_BLOCKS * std::max(B, 1), s));
    CK(cudaMemsetAsync(dv.fx, 0, sizeof(long long) * 6 * std::max(B, 1), s));
    CK(cudaMemsetAsync(dv.fi, 0, sizeof(int) * 6 * std::max(B, 1), s));
    CK(cudaMemsetAsync(dv.geom, 0, sizeof(lbm::BodyGeom) * 2 * std::max(B, 1), s));
    // stamps that match no state (q = 0 is no unit quaternion): the first
    // step computes every geometry record
    CK(cudaMemsetAsync(dv.gstamp, 0, sizeof(BodyState) * 2 * std::max(B, 1), s));
    CK(cudaMemsetAsync(dv.bcount, 0, sizeof(int) * 4, s));
    CK(cudaMemsetAsync(dv.blocks_done, 0, sizeof(unsigned) * 4, s));
    CK(cudaMemsetAsync(dv.body_done, 0, sizeof(unsigned) * std::max(B, 1), s));
    if (!spring_list.empty())
        CK(cudaMemcpyAsync(slist, spring_list.data(), sizeof(int) * spring_list.size(), cudaMemcpyHostToDevice, s));
    CK(cudaMemsetAsync(dv.seg_count, 0, sizeof(int) * std::max(B, 1) * dv.link_side, s));
    const int st[4] = {0, 0, 1, 0};           // status, pad, changed[0] = 1, changed[1] = 0
    CK(cudaMemcpyAsync(dv.status, st, sizeof st, cudaMemcpyHostToDevice, s));
    const long long t0 = 0;
    CK(cudaMemcpyAsync(dv.t_dev, &t0, sizeof t0, cudaMemcpyHostToDevice, s));
    CK(cudaMemsetAsync(dv.tstep, 0, sizeof(long long) * 2, s));
    CK(cudaMemsetAsync(dv.near_count, 0, sizeof(int) * 2, s));
    for (int i = 0; i < 2; ++i)
        CK(cudaMemsetAsync(dv.near_mask[i], 0,
                           sizeof(unsigned) * (dv.overlap ? (size_t)lbm::near_tile_count(dv) : 1), s));
    CK(cudaMemsetAsync(h->tape.ctl, 0, sizeof(lbm::TapeCtl), s));
    if (B) CK(cudaMemcpyAsync(props, props_h.data(), sizeof(BodyProps) * B, cudaMemcpyHostToDevice, s));
    if (!h->springs.empty())
        CK(cudaMemcpyAsync(springs, h->springs.data(), sizeof(Spring) * h->springs.size(), cudaMemcpyHostToDevice, s));
    if (!drives_h.empty())
        CK(cudaMemcpyAsync(drives, drives_h.data(), sizeof(DriveTerm) * drives_h.size(), cudaMemcpyHostToDevice, s));
    // the staging vectors above go out of scope: finish the copies first
    CK(cudaStreamSynchronize(s));
    if ((rc = upload_bodies(h))) return rc;
    if ((rc = init_flags(h))) return rc;
    CK(cudaStreamSynchronize(s));
    h->ready = true;
    return LBM_OK;
}

int build_graphs(lbm_t *h) {
    if (h->graphs_ready) return LBM_OK;
    // overlapped steps: the chain (captured on cap) takes precedence over the
    // far bulk kernel, so that its short kernels start as soon as SMs free
    const bool ov = h->dv.overlap != 0;
    int least = 0, greatest = 0;
    CK(cudaDeviceGetStreamPriorityRange(&least, &greatest));
    if (!h->cap) CK(cudaStreamCreateWithPriority(&h->cap, cudaStreamNonBlocking, ov ? greatest : 0));
    if (!h->side) CK(cudaStreamCreateWithFlags(&h->side, cudaStreamNonBlocking));
    if (!h->fork_ev) CK(cudaEventCreateWithFlags(&h->fork_ev, cudaEventDisableTiming));
    if (!h->join_ev) CK(cudaEventCreateWithFlags(&h->join_ev, cudaEventDisableTiming));
    if (!h->side2) CK(cudaStreamCreateWithFlags(&h->side2, cudaStreamNonBlocking));
    if (!h->join2_ev) CK(cudaEventCreateWithFlags(&h->join2_ev, cudaEventDisableTiming));
    if (ov) {
        if (!h->far) CK(cudaStreamCreateWithPriority(&h->far, cudaStreamNonBlocking, least));
        for (int i = 0; i < 2; ++i) {
            if (!h->far_ev[i]) CK(cudaEventCreateWithFlags(&h->far_ev[i], cudaEventDisableTiming));
            if (!h->near_ev[i]) CK(cudaEventCreateWithFlags(&h->near_ev[i], cudaEventDisableTiming));
        }
    }
    // steps p0, p0 + 1, ... of a graph; the far stream joins back at the end
    auto steps = [&](int p0, int n) {
        for (int i = 0; i < n; ++i) {
            const int p = (p0 + i) & 1;
            if (ov) enqueue_overlapped(h, p, h->cap, i == 0);
            else enqueue_step(h, p, h->cap, nullptr, nullptr, true, false);
        }
        if (ov) cudaStreamWaitEvent(h->cap, h->far_ev[(p0 + n - 1) & 1], 0);
    };
    // one graph of n steps from parity p0
    auto capture = [&](int p0, int n, cudaGraphExec_t *x) {
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return e;
        steps(p0, n);
        e = cudaStreamEndCapture(h->cap, &g);
        if (e == cudaSuccess) e = cudaGraphInstantiate(x, g, ov ? cudaGraphInstantiateFlagUseNodePriority : 0);
        if (g) cudaGraphDestroy(g);
        return e;
    };
    // with LBM_DEBUG_NO_PDL 0, serial steps launch the force kernel and the
    // next step's remap programmatically dependent on the kernel before them
    // in the chain, so that their blocks are resident, waiting, when the bulk
    // kernel and the force kernel end (overlapped steps order their streams
    // by events and node priorities instead)
    h->dv.pdl = !ov && !h->no_pdl;
    cudaError_t e = capture(0, 1, &h->single[0]);
    if (e == cudaSuccess) e = capture(1, 1, &h->single[1]);
    if (e == cudaSuccess) e = capture(0, CHUNK_STEPS, &h->chunk);
    h->dv.pdl = 0;
    if (e != cudaSuccess) {
        drop_graphs(h);
        return cuda_fail(h, e, "capture of the step graphs");
    }
    h->graphs_ready = true;
    return LBM_OK;
}

int status_error(lbm_t *h, int st) {
    // a step cut short (a wait that ran out, a full list) comes first: the
    // other bits may be its consequences
    if (st & lbm::ST_TIMEOUT) return fail(h, LBM_E_TIMEOUT, "a bounded wait on a bulk copy ran out");
    if (st & lbm::ST_LINKS) return fail(h, LBM_E_LINKS, "link or boundary-cell list capacity exceeded");
    if (st & lbm::ST_NAN) return fail(h, LBM_E_NAN, "non-finite body state or link term");
    if (st & lbm::ST_OVERLAP) return fail(h, LBM_E_OVERLAP, "two bodies cover the same cell");
    if (st & lbm::ST_OUTSIDE) return fail(h, LBM_E_OUTSIDE, "a body crosses a wall of the domain");
    if (st & lbm::ST_UNSTABLE)
        return fail(h, LBM_E_UNSTABLE, "a body moved more than %g lattice units in one step", LBM_MAX_BODY_STEP);
    return LBM_OK;
}

int check_status(lbm_t *h) {
    int st = 0;
    CK(cudaMemcpy(&st, h->dv.status, sizeof st, cudaMemcpyDeviceToHost));
    return status_error(h, st);
}

int sync_and_check(lbm_t *h) {
    if (!h->ready) return LBM_OK;
    CK(cudaStreamSynchronize(h->stream));
    if (h->rd_stream) CK(cudaStreamSynchronize(h->rd_stream));
    CK(cudaGetLastError());
    return check_status(h);
}

void release_device(lbm_t *h) {
    if (h->ready) cudaStreamSynchronize(h->stream);
    if (h->rd_stream) {
        cudaStreamSynchronize(h->rd_stream);
        cudaStreamDestroy(h->rd_stream);
        h->rd_stream = nullptr;
    }
    if (h->rd_after) cudaEventDestroy(h->rd_after);
    h->rd_after = nullptr;
    h->rd_pending[0] = h->rd_pending[1] = -1;
    for (cudaEvent_t &ev : h->rd_ev)
        if (ev) {
            cudaEventDestroy(ev);
            ev = nullptr;
        }
    if (h->rd_status) cudaFreeHost(h->rd_status);
    h->rd_status = nullptr;
    for (int p = 0; p < 2; ++p)
        if (h->single[p]) cudaGraphExecDestroy(h->single[p]);
    if (h->chunk) cudaGraphExecDestroy(h->chunk);
    if (h->cap) cudaStreamDestroy(h->cap);
    if (h->side) cudaStreamDestroy(h->side);
    if (h->fork_ev) cudaEventDestroy(h->fork_ev);
    if (h->join_ev) cudaEventDestroy(h->join_ev);
    if (h->side2) cudaStreamDestroy(h->side2);
    if (h->join2_ev) cudaEventDestroy(h->join2_ev);
    if (h->far) cudaStreamDestroy(h->far);
    for (int i = 0; i < 2; ++i) {
        if (h->far_ev[i]) cudaEventDestroy(h->far_ev[i]);
        if (h->near_ev[i]) cudaEventDestroy(h->near_ev[i]);
    }
    for (void *p : h->tape.allocs) dfree(h, p);
    h->tape.allocs.clear();
    for (void *p : h->allocs) dfree(h, p);
    h->allocs.clear();
}

// ---- reverse sweep helpers ---------------------------------------------------

template <typename T>
int alloc_list(lbm_t *h, std::vector<void *> &list, T **out, size_t bytes) {
    void *p = dalloc(h, bytes);
    if (!p) return fail(h, LBM_E_OOM, "device allocation of %zu bytes failed", bytes);
    list.push_back(p);
    *out = static_cast<T *>(p);
    return LBM_OK;
}

void free_list(lbm_t *h, std::vector<void *> &list) {
    for (void *p : list) dfree(h, p);
    list.clear();
}

size_t adj_bytes(int precision) { return precision == LBM_PREC_F64 ? 8 : 4; }

int last_parity(const lbm_t *h) { return (int)((h->steps + 1) & 1); }

}  // namespace

// the library is built with hidden visibility; only the C ABI is exported
#pragma GCC visibility push(default)
extern "C" {

int lbm_create_ex(int nx, int ny, int nz, double tau, int bc, int precision, const double g[3],
                  int options, lbm_t **out) {
    if (!out) return LBM_E_ARG;
    *out = nullptr;
    if (nx < 1 || ny < 1 || nz < 1 || !(tau > 0.5) || bc < 0 || bc > 7 || precision < 0 || precision > 3 ||
        (options & ~(LBM_OPT_NO_FLUID | LBM_OPT_AVERAGE_FORCE | LBM_OPT_OVERLAP)))
        return LBM_E_ARG;
    const long long C = (long long)nx * ny * nz;
    if (C > (1LL << 31) - 1) return LBM_E_ARG;   // link cells are 32-bit indices
    lbm_t *h = new (std::nothrow) lbm_s();
    if (!h) return LBM_E_OOM;
    h->nx = nx; h->ny = ny; h->nz = nz; h->bc = bc; h->tau = tau;
    h->precision = precision; h->options = options; h->C = C;
    if (g)
        for (int i = 0; i < 3; ++i) h->g[i] = g[i];
    *out = h;
    return LBM_OK;
}

int lbm_create(int nx, int ny, int nz, double tau, int bc, lbm_t **out) {
    return lbm_create_ex(nx, ny, nz, tau, bc, LBM_PREC_F32, nullptr, 0, out);
}

int lbm_destroy(lbm_t *h) {
    if (!h) return LBM_OK;
    release_device(h);
    delete h;
    return LBM_OK;
}

int lbm_set_allocator(lbm_t *h, lbm_alloc_fn a, lbm_free_fn f, void *ctx) {
    if (!h) return LBM_E_ARG;
    if (h->ready) return fail(h, LBM_E_STATE, "allocator must be set before the first device allocation");
    if ((a == nullptr) != (f == nullptr)) return fail(h, LBM_E_ARG, "allocator needs both functions");
    h->afn = a; h->ffn = f; h->actx = ctx;
    return LBM_OK;
}

int lbm_set_stream(lbm_t *h, void *stream) {
    if (!h) return LBM_E_ARG;
    h->stream = static_cast<cudaStream_t>(stream);
    return LBM_OK;
}

namespace {
// Volume and body-frame principal moments of inertia of a uniform solid
// sphere, or capsule (cylinder of length l along the body x axis plus two
// hemispherical caps), and their derivatives with respect to the mass and
// the cylinder length: q = (V, I1, I2, I3).
void body_properties(int shape, double r, double l, double m, double q[4], double dq_dm[4], double dq_dl[4]) {
    if (shape == LBM_SHAPE_SPHERE) {
        q[0] = 4.0 / 3.0 * M_PI * r * r * r;
        dq_dm[0] = dq_dl[0] = 0.0;
        for (int i = 1; i < 4; ++i) {
            q[i] = 0.4 * m * r * r;
            dq_dm[i] = 0.4 * r * r;
            dq_dl[i] = 0.0;
        }
        return;
    }
    // I = m N / V with N the volume-weighted moment per unit density:
    // cylinder (mass m vc / V) and two caps (m vh / V each), the caps'
    // centroids 3r/8 beyond the cylinder's ends
    const double vc = M_PI * r * r * l, vh = 2.0 / 3.0 * M_PI * r * r * r;
    const double V = vc + 2.0 * vh, dV = M_PI * r * r;
    const double N1 = vc * 0.5 * r * r + 2.0 * vh * 0.4 * r * r;
    const double dN1 = dV * 0.5 * r * r;
    const double N2 = vc * (r * r / 4.0 + l * l / 12.0) + 2.0 * vh * (0.4 * r * r + l * l / 4.0 + 3.0 * l * r / 8.0);
    const double dN2 = dV * (r * r / 4.0 + l * l / 12.0) + vc * (l / 6.0) + 2.0 * vh * (l / 2.0 + 3.0 * r / 8.0);
    q[0] = V;
    dq_dm[0] = 0.0;
    dq_dl[0] = dV;
    const double N[2] = {N1, N2}, dN[2] = {dN1, dN2};
    for (int i = 1; i < 4; ++i) {
        const int k = i == 1 ? 0 : 1;
        q[i] = m * N[k] / V;
        dq_dm[i] = N[k] / V;
        dq_dl[i] = m * (dN[k] * V - N[k] * dV) / (V * V);
    }
}
}  // namespace

int lbm_body_properties(int shape, double radius, double length, double mass, double out[4], double d_mass[4],
                        double d_length[4]) {
    if (!out || (shape != LBM_SHAPE_SPHERE && shape != LBM_SHAPE_CAPSULE) || !(radius > 0) || !(mass > 0) ||
        !(length >= 0) || (shape == LBM_SHAPE_SPHERE && length != 0))
        return LBM_E_ARG;
    double q[4], dm[4], dl[4];
    body_properties(shape, radius, length, mass, q, dm, dl);
    for (int i = 0; i < 4; ++i) {
        out[i] = q[i];
        if (d_mass) d_mass[i] = dm[i];
        if (d_length) d_length[i] = dl[i];
    }
    return LBM_OK;
}

int lbm_add_body(lbm_t *h, int shape, double radius, double length, double mass, const double pos[3],
                 const double orient[4]) {
    if (!h || !pos) return fail(h, LBM_E_ARG, "lbm_add_body: null position");
    if (h->ready) return fail(h, LBM_E_STATE, "bodies must be added before the first step");
    if ((int)h->props.size() >= LBM_MAX_BODIES) return fail(h, LBM_E_ARG, "at most %d bodies", LBM_MAX_BODIES);
    if (shape != LBM_SHAPE_SPHERE && shape != LBM_SHAPE_CAPSULE) return fail(h, LBM_E_ARG, "unknown shape");
    if (!(radius > 0) || !(mass > 0) || !(length >= 0) || (shape == LBM_SHAPE_SPHERE && length != 0) ||
        !(radius + 0.5 * length < 500.0))
        return fail(h, LBM_E_ARG, "bad body dimensions");
    for (int i = 0; i < 3; ++i)
        if (!std::isfinite(pos[i])) return fail(h, LBM_E_ARG, "non-finite position");
    BodyProps p{};
    p.shape = shape; p.r = radius; p.l = length; p.m = mass;
    p.E = (int)std::ceil(radius + 0.5 * length) + 1;
    if (fluid(h)) {
        // the remap and link scans wrap their cubes on periodic axes: a cube
        // longer than the axis would visit cells twice and count their links
        // twice
        const int side = 2 * (p.E + lbm::REMAP_MARGIN) + 1;
        const int n[3] = {h->nx, h->ny, h->nz};
        for (int i = 0; i < 3; ++i)
            if (((h->bc >> i) & 1) && n[i] < side)
                return fail(h, LBM_E_ARG,
                            "periodic extent %d along axis %d is shorter than the body's remap cube (side %d)", n[i],
                            i, side);
    }
    p.reach = radius + 0.5 * length;
    p.r2f = (float)(radius * radius);
    p.hf = (float)(0.5 * length);
    // the FP32 inside test's margin: its error stays near 1e-5 max(r^2, 1)
    // and grows like 1.3e-7 l r for long thin capsules
    p.marginf = (float)std::max(1e-3 * std::max(radius * radius, 1.0), 2e-6 * length * std::max(radius, 1.0));
    {
        double q[4], dm[4], dl[4];
        body_properties(shape, radius, length, mass, q, dm, dl);
        p.volume = q[0];
        for (int i = 0; i < 3; ++i) p.inertia[i] = q[1 + i];
    }
    BodyState s{};
    for (int i = 0; i < 3; ++i) s.X[i] = pos[i];
    if (orient) {
        const double n = std::sqrt(orient[0] * orient[0] + orient[1] * orient[1] + orient[2] * orient[2] +
                                   orient[3] * orient[3]);
        if (!(n > 0)) return fail(h, LBM_E_ARG, "zero quaternion");
        for (int i = 0; i < 4; ++i) s.q[i] = orient[i] / n;
    } else {
        s.q[0] = 1.0;
    }
    h->props.push_back(p);
    h->init_state.push_back(s);
    return (int)h->props.size() - 1;
}

int lbm_add_spring(lbm_t *h, int i, int j, double k, double rest, double damping) {
    if (!h) return LBM_E_ARG;
    if (h->ready) return fail(h, LBM_E_STATE, "springs must be added before the first step");
    const int B = nb(h);
    if (i < 0 || j < 0 || i >= B || j >= B || i == j || !(k >= 0) || !(rest >= 0) || !(damping >= 0))
        return fail(h, LBM_E_ARG, "bad spring");
    h->springs.push_back(Spring{i, j, k, rest, damping});
    return (int)h->springs.size() - 1;
}

int lbm_set_drive(lbm_t *h, int body, double amp, double freq, double phase) {
    if (!h) return LBM_E_ARG;
    if (h->ready) return fail(h, LBM_E_STATE, "drives must be added before the first step");
    if (body < 0 || body >= nb(h) || !(freq > 0) || !(phase >= 0) || !std::isfinite(amp))
        return fail(h, LBM_E_ARG, "bad drive");
    h->drives.push_back(DriveTerm{body, amp, freq, phase, INFINITY, 0.0, 0.0, {1.0, 0.0, 0.0}});
    return (int)h->drives.size() - 1;
}

int lbm_set_drive_axis(lbm_t *h, int term, const double axis[3]) {
    if (!h || !axis || term < 0 || term >= (int)h->drives.size())
        return fail(h, LBM_E_ARG, "lbm_set_drive_axis: no drive term %d, or a null axis", term);
    if (h->ready) return fail(h, LBM_E_STATE, "drive axes must be set before the first step");
    for (int i = 0; i < 3; ++i) {
        if (!std::isfinite(axis[i])) return fail(h, LBM_E_ARG, "non-finite drive axis");
        h->drives[term].axis[i] = axis[i];
    }
    return LBM_OK;
}

int lbm_set_drive_window(lbm_t *h, int term, double t_off) {
    if (!h || term < 0 || term >= (int)h->drives.size())
        return fail(h, LBM_E_ARG, "lbm_set_drive_window: no drive term %d", term);
    if (h->ready) return fail(h, LBM_E_STATE, "drive windows must be set before the first step");
    h->drives[term].t_off = t_off;
    return LBM_OK;
}

int lbm_set_body_state(lbm_t *h, int b, const double state[13]) {
    if (!h || !state || b < 0 || b >= nb(h))
        return fail(h, LBM_E_ARG, "lbm_set_body_state: no body %d, or a null state", b);
    BodyState s;
    std::memcpy(&s, state, sizeof s);
    const double n = std::sqrt(s.q[0] * s.q[0] + s.q[1] * s.q[1] + s.q[2] * s.q[2] + s.q[3] * s.q[3]);
    if (!(n > 0)) return fail(h, LBM_E_ARG, "zero quaternion");
    for (int i = 0; i < 4; ++i) s.q[i] /= n;
    if (!h->ready || h->steps == 0) {
        h->init_state[b] = s;
        if (!h->ready) return LBM_OK;
        int rc;
        if ((rc = upload_bodies(h))) return rc;
        if ((rc = init_flags(h))) return rc;
        CK(cudaStreamSynchronize(h->stream));
        return LBM_OK;
    }
    int rc = sync_and_check(h);
    if (rc) return rc;
    BodyState *cur = h->bodies[h->steps & 1] + b;
    BodyState old;
    CK(cudaMemcpy(&old, cur, sizeof old, cudaMemcpyDeviceToHost));
    for (int i = 0; i < 3; ++i)
        if (!(std::fabs(s.X[i] - old.X[i]) < LBM_MAX_BODY_STEP))
            return fail(h, LBM_E_STATE, "after the first step a body may move by less than %g per axis",
                        LBM_MAX_BODY_STEP);
    CK(cudaMemcpy(cur, &s, sizeof s, cudaMemcpyHostToDevice));
    h->tiles_stale = true;
    h->need_prep = true;
    return LBM_OK;
}

int lbm_set_fields(lbm_t *h, int what, const void *in, int dtype) {
    if (!h || !in) return fail(h, LBM_E_ARG, "lbm_set_fields: null input");
    if (what != LBM_FIELD_POP || dtype != LBM_DTYPE_F64)
        return fail(h, LBM_E_ARG, "only LBM_FIELD_POP as LBM_DTYPE_F64 can be set");
    int rc = ensure_device(h);
    if (rc) return rc;
    if ((rc = sync_and_check(h))) return rc;
    const size_t bytes = sizeof(double) * lbm::Q * h->C;
    double *tmp = static_cast<double *>(dalloc(h, bytes));
    if (!tmp) return fail(h, LBM_E_OOM, "device allocation of %zu bytes failed", bytes);
    cudaError_t e = cudaMemcpyAsync(tmp, in, bytes, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) {
        lbm::launch_import_pop(h->dv, h->pop[last_parity(h)], tmp, h->stream);
        e = cudaStreamSynchronize(h->stream);
    }
    dfree(h, tmp);
    if (e != cudaSuccess) return cuda_fail(h, e, "lbm_set_fields");
    return LBM_OK;
}

// before steps that write body buffer p: wait (on the handle's stream) for a
// pending asynchronous read of it
static int wait_read(lbm_t *h, int p) {
    if (h->rd_pending[p] >= 0) {
        CK(cudaStreamWaitEvent(h->stream, h->rd_ev[h->rd_pending[p]], 0));
        h->rd_pending[p] = -1;
    }
    return LBM_OK;
}

int lbm_step(lbm_t *h, int n) {
    if (!h || n < 0) return fail(h, LBM_E_ARG, "lbm_step: negative step count %d", n);
    int rc = ensure_device(h);
    if (rc) return rc;
    if ((rc = build_graphs(h))) return rc;
    if (n > 0 && (rc = refresh_tiles(h))) return rc;
    if (n > 0 && h->need_prep && nb(h) > 0 && fluid(h) && !overlapped(h)) {
        // the step graphs leave the body preparation out: it runs here after
        // the host wrote a state (creation, lbm_set_body_state, lbm_load, a
        // reverse sweep's recomputation)
        lbm::launch_prep(h->dv, step_ptrs(h, (int)(h->steps & 1)), h->stream);
        CK(cudaGetLastError());
    }
    if (n > 0) h->need_prep = false;
    while (n > 0) {
        const int p = (int)(h->steps & 1);
        if (p == 0 && n >= CHUNK_STEPS) {
            if ((rc = wait_read(h, 0)) || (rc = wait_read(h, 1))) return rc;
            CK(cudaGraphLaunch(h->chunk, h->stream));
            h->steps += CHUNK_STEPS;
            n -= CHUNK_STEPS;
        } else {
            if ((rc = wait_read(h, p ^ 1))) return rc;      // the step writes state n + 1 into buffer p ^ 1
            CK(cudaGraphLaunch(h->single[p], h->stream));
            h->steps += 1;
            n -= 1;
        }
    }
    return LBM_OK;
}

int lbm_sync(lbm_t *h) {
    if (!h) return LBM_E_ARG;
    return sync_and_check(h);
}

int lbm_average_begin(lbm_t *h) {
    if (!h) return LBM_E_ARG;
    if (!fluid(h)) return fail(h, LBM_E_STATE, "no fluid to average");
    int rc = ensure_device(h);
    if (rc) return rc;
    if ((rc = sync_and_check(h))) return rc;
    if (!h->avg_sum) {
        if ((rc = alloc_into(h, &h->avg_sum, sizeof(double) * 3 * (size_t)h->C))) return rc;
        if ((rc = alloc_into(h, &h->avg_count, sizeof(long long)))) return rc;
    }
    CK(cudaMemsetAsync(h->avg_sum, 0, sizeof(double) * 3 * (size_t)h->C, h->stream));
    CK(cudaMemsetAsync(h->avg_count, 0, sizeof(long long), h->stream));
    if (!h->dv.avg_u) {
        h->dv.avg_u = h->avg_sum;
        h->dv.avg_n = h->avg_count;
        drop_graphs(h);
    }
    return LBM_OK;
}

int lbm_average_stop(lbm_t *h) {
    if (!h) return LBM_E_ARG;
    if (h->dv.avg_u) {
        h->dv.avg_u = nullptr;
        h->dv.avg_n = nullptr;
        drop_graphs(h);
    }
    return LBM_OK;
}

int lbm_average_get(lbm_t *h, double *out, long long *steps) {
    if (!h || !out) return fail(h, LBM_E_ARG, "lbm_average_get: null output");
    if (!h->avg_sum) return fail(h, LBM_E_STATE, "no average was begun");
    int rc = sync_and_check(h);
    if (rc) return rc;
    long long n = 0;
    CK(cudaMemcpy(&n, h->avg_count, sizeof n, cudaMemcpyDeviceToHost));
    const size_t count = 3 * (size_t)h->C;
    CK(cudaMemcpy(out, h->avg_sum, sizeof(double) * count, cudaMemcpyDeviceToHost));
    if (n > 0)
        for (size_t i = 0; i < count; ++i) out[i] /= (double)n;
    if (steps) *steps = n;
    return LBM_OK;
}

long long lbm_steps_done(lbm_t *h) { return h ? h->steps : -1; }

int lbm_get_bodies(lbm_t *h, double *out) {
    if (!h || !out) return fail(h, LBM_E_ARG, "lbm_get_bodies: null output");
    if (!h->ready) {
        std::memcpy(out, h->init_state.data(), sizeof(BodyState) * nb(h));
        return LBM_OK;
    }
    int rc = sync_and_check(h);
    if (rc) return rc;
    if (nb(h)) CK(cudaMemcpy(out, h->bodies[h->steps & 1], sizeof(BodyState) * nb(h), cudaMemcpyDeviceToHost));
    return LBM_OK;
}

int lbm_get_bodies_async(lbm_t *h, double *out, long long *ticket) {
    if (!h || !out || !ticket) return fail(h, LBM_E_ARG, "lbm_get_bodies_async: null output or ticket");
    *ticket = -1;
    if (!h->ready) {
        std::memcpy(out, h->init_state.data(), sizeof(BodyState) * nb(h));
        return LBM_OK;
    }
    if (!h->rd_status) {
        CK(cudaHostAlloc(reinterpret_cast<void **>(&h->rd_status), sizeof(int) * lbm_s::READS, cudaHostAllocDefault));
        for (cudaEvent_t &ev : h->rd_ev) CK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
        CK(cudaStreamCreateWithFlags(&h->rd_stream, cudaStreamNonBlocking));
        CK(cudaEventCreateWithFlags(&h->rd_after, cudaEventDisableTiming));
    }
    const int slot = (int)(h->rd_seq % lbm_s::READS);
    const int buf = (int)(h->steps & 1);
    // after the steps enqueued so far, on the read stream: the next step
    // reads this buffer and writes the other one, so it runs beside the copy
    cudaStream_t s = h->rd_stream;
    CK(cudaEventRecord(h->rd_after, h->stream));
    CK(cudaStreamWaitEvent(s, h->rd_after, 0));
    if (nb(h))
        CK(cudaMemcpyAsync(out, h->bodies[buf], sizeof(BodyState) * nb(h), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(h->rd_status + slot, h->dv.status, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaEventRecord(h->rd_ev[slot], s));
    h->rd_pending[buf] = slot;
    *ticket = h->rd_seq++;
    return LBM_OK;
}

int lbm_wait_ticket(lbm_t *h, long long ticket) {
    if (!h || ticket >= h->rd_seq) return h ? fail(h, LBM_E_ARG, "no read with ticket %lld", ticket) : LBM_E_ARG;
    if (ticket < 0) return LBM_OK;
    // a slot re-recorded by a later read completes after this one
    const int slot = (int)(ticket % lbm_s::READS);
    CK(cudaEventSynchronize(h->rd_ev[slot]));
    CK(cudaGetLastError());
    return status_error(h, h->rd_status[slot]);
}

int lbm_get_forces(lbm_t *h, double *out) {
    if (!h || !out) return fail(h, LBM_E_ARG, "lbm_get_forces: null output");
    if (!h->ready) {
        std::memset(out, 0, sizeof(double) * 6 * nb(h));
        return LBM_OK;
    }
    int rc = sync_and_check(h);
    if (rc) return rc;
    if (nb(h)) CK(cudaMemcpy(out, h->dv.fh, sizeof(double) * 6 * nb(h), cudaMemcpyDeviceToHost));
    return LBM_OK;
}

static size_t field_elems(const lbm_t *h, int what) {
    return (size_t)h->C * (what == LBM_FIELD_U ? 3 : (what == LBM_FIELD_POP ? lbm::Q : 1));
}

static int check_field_args(lbm_t *h, int what, int dtype) {
    if (what < 0 || what > 3) return fail(h, LBM_E_ARG, "unknown field");
    if (what == LBM_FIELD_FLAGS ? dtype != LBM_DTYPE_U8 : (dtype != LBM_DTYPE_F64 && dtype != LBM_DTYPE_F32))
        return fail(h, LBM_E_ARG, "unsupported dtype for this field");
    return LBM_OK;
}

int lbm_get_fields_device(lbm_t *h, int what, void *dev_out, int dtype) {
    if (!h || !dev_out) return fail(h, LBM_E_ARG, "lbm_get_fields_device: null output");
    int rc = check_field_args(h, what, dtype);
    if (rc) return rc;
    if ((rc = ensure_device(h))) return rc;
    const int p = last_parity(h);
    if (what == LBM_FIELD_FLAGS && h->steps == 0) {
        CK(cudaMemsetAsync(dev_out, 0, (size_t)h->C, h->stream));
        return LBM_OK;
    }
    lbm::launch_export(h->dv, h->pop[p], h->flags[p], h->bid[p], what, h->steps > 0 ? 1 : 0, dev_out, dtype,
                       h->stream);
    CK(cudaGetLastError());
    return LBM_OK;
}

int lbm_get_fields(lbm_t *h, int what, void *out, int dtype) {
    if (!h || !out) return fail(h, LBM_E_ARG, "lbm_get_fields: null output");
    int rc = check_field_args(h, what, dtype);
    if (rc) return rc;
    if ((rc = ensure_device(h))) return rc;
    if ((rc = sync_and_check(h))) return rc;
    const size_t es = what == LBM_FIELD_FLAGS ? 1 : (dtype == LBM_DTYPE_F32 ? 4 : 8);
    const size_t bytes = field_elems(h, what) * es;
    void *tmp = dalloc(h, bytes);
    if (!tmp) return fail(h, LBM_E_OOM, "device allocation of %zu bytes failed", bytes);
    rc = lbm_get_fields_device(h, what, tmp, dtype);
    cudaError_t e = cudaSuccess;
    if (!rc) {
        e = cudaMemcpyAsync(out, tmp, bytes, cudaMemcpyDeviceToHost, h->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    }
    dfree(h, tmp);
    if (rc) return rc;
    if (e != cudaSuccess) return cuda_fail(h, e, "lbm_get_fields");
    return LBM_OK;
}

int lbm_enable_history(lbm_t *h, int capacity) {
    if (!h || capacity < 0) return fail(h, LBM_E_ARG, "lbm_enable_history: negative capacity");
    if (h->ready) return fail(h, LBM_E_STATE, "history must be enabled before the first step");
    h->hist_cap = capacity;
    return LBM_OK;
}

int lbm_get_history(lbm_t *h, double *out, int max_steps, int *n_out) {
    if (!h || !out || !n_out || max_steps < 0)
        return fail(h, LBM_E_ARG, "lbm_get_history: null output or negative max_steps");
    *n_out = 0;
    if (!h->ready || h->hist_cap == 0 || nb(h) == 0) return LBM_OK;
    int rc = sync_and_check(h);
    if (rc) return rc;
    const long long n = std::min<long long>(std::min<long long>(h->steps, h->hist_cap), max_steps);
    const size_t per = (size_t)13 * nb(h);
    std::vector<double> ring(per * h->hist_cap);
    CK(cudaMemcpy(ring.data(), h->dv.hist, sizeof(double) * ring.size(), cudaMemcpyDeviceToHost));
    for (long long i = 0; i < n; ++i) {
        const long long t = h->steps - n + i;           // step whose result is state t + 1
        std::memcpy(out + i * per, ring.data() + (t % h->hist_cap) * per, sizeof(double) * per);
    }
    *n_out = (int)n;
    return LBM_OK;
}

namespace {
struct SaveHeader {
    char magic[8];
    int nx, ny, nz, precision, nb, pad;
    long long steps;
};
}  // namespace

int lbm_save(lbm_t *h, const char *path) {
    if (!h || !path) return fail(h, LBM_E_ARG, "lbm_save: null path");
    int rc = ensure_device(h);
    if (rc) return rc;
    if ((rc = sync_and_check(h))) return rc;
    FILE *f = std::fopen(path, "wb");
    if (!f) return fail(h, LBM_E_ARG, "cannot open %s", path);
    SaveHeader hd{};
    std::memcpy(hd.magic, SAVE_MAGIC, 8);
    hd.nx = h->nx; hd.ny = h->ny; hd.nz = h->nz; hd.precision = h->precision; hd.nb = nb(h);
    hd.steps = h->steps;
    bool ok = std::fwrite(&hd, sizeof hd, 1, f) == 1;
    const size_t pb = pop_bytes(h->precision) * lbm::Q * h->C;
    std::vector<char> buf(std::max<size_t>(pb, 64));
    auto put = [&](const void *dev, size_t bytes) {
        if (!ok) return;
        if (cudaMemcpy(buf.data(), dev, bytes, cudaMemcpyDeviceToHost) != cudaSuccess) { ok = false; return; }
        ok = std::fwrite(buf.data(), 1, bytes, f) == bytes;
    };
    put(h->pop[last_parity(h)], pb);
    for (int i = 0; i < 2; ++i) { put(h->flags[i], h->C); put(h->bid[i], h->C); }
    if (nb(h)) {
        for (int i = 0; i < 2; ++i) put(h->bodies[i], sizeof(BodyState) * nb(h));
        put(h->dv.fh, sizeof(double) * 6 * nb(h));
    }
    put(h->dv.t_dev, sizeof(long long));
    ok = (std::fclose(f) == 0) && ok;
    return ok ? LBM_OK : fail(h, LBM_E_ARG, "writing %s failed", path);
}

int lbm_load(lbm_t *h, const char *path) {
    if (!h || !path) return fail(h, LBM_E_ARG, "lbm_load: null path");
    int rc = ensure_device(h);
    if (rc) return rc;
    if ((rc = sync_and_check(h))) return rc;
    FILE *f = std::fopen(path, "rb");
    if (!f) return fail(h, LBM_E_ARG, "cannot open %s", path);
    SaveHeader hd{};
    bool ok = std::fread(&hd, sizeof hd, 1, f) == 1 && std::memcmp(hd.magic, SAVE_MAGIC, 8) == 0 &&
              hd.nx == h->nx && hd.ny == h->ny && hd.nz == h->nz && hd.precision == h->precision &&
              hd.nb == nb(h);
    if (!ok) {
        std::fclose(f);
        return fail(h, LBM_E_ARG, "%s does not match this lattice", path);
    }
    h->steps = hd.steps;
    const size_t pb = pop_bytes(h->precision) * lbm::Q * h->C;
    std::vector<char> buf(std::max<size_t>(pb, 64));
    auto get = [&](void *dev, size_t bytes) {
        if (!ok) return;
        ok = std::fread(buf.data(), 1, bytes, f) == bytes &&
             cudaMemcpy(dev, buf.data(), bytes, cudaMemcpyHostToDevice) == cudaSuccess;
    };
    get(h->pop[last_parity(h)], pb);
    for (int i = 0; i < 2; ++i) { get(h->flags[i], h->C); get(h->bid[i], h->C); }
    if (nb(h)) {
        for (int i = 0; i < 2; ++i) get(h->bodies[i], sizeof(BodyState) * nb(h));
        get(h->dv.fh, sizeof(double) * 6 * nb(h));
    }
    get(h->dv.t_dev, sizeof(long long));
    std::fclose(f);
    if (!ok) return fail(h, LBM_E_ARG, "reading %s failed", path);
    // the next step rebuilds its link lists from the restored flags, and
    // its near tiles from the restored states
    const int st[4] = {0, 0, 1, 1};
    CK(cudaMemcpy(h->dv.status, st, sizeof st, cudaMemcpyHostToDevice));
    h->tiles_stale = true;
    h->need_prep = true;
    return LBM_OK;
}

int lbm_time_kernels(lbm_t *h, int n, double *ms_out, int slots) {
    if (!h || n < 0 || !ms_out || slots < 0)
        return fail(h, LBM_E_ARG, "lbm_time_kernels: negative count, null output or negative slots");
    int rc = ensure_device(h);
    if (rc) return rc;
    if ((rc = sync_and_check(h))) return rc;
    double total[LBM_NUM_KERNELS] = {0, 0, 0, 0, 0, 0};
    cudaEvent_t ev[2 * LBM_NUM_KERNELS];
    for (auto &e : ev) CK(cudaEventCreate(&e));
    for (int it = 0; it < n; ++it) {
        bool ran[LBM_NUM_KERNELS] = {false, false, false, false, false, false};
        enqueue_step(h, (int)(h->steps & 1), h->stream, ev, ran);
        h->steps += 1;
        h->tiles_stale = true;              // steps without the overlapped graphs
        CK(cudaStreamSynchronize(h->stream));
        for (int k = 0; k < LBM_NUM_KERNELS; ++k) {
            if (!ran[k]) continue;
            float ms = 0;
            CK(cudaEventElapsedTime(&ms, ev[2 * k], ev[2 * k + 1]));
            total[k] += ms;
        }
    }
    for (auto &e : ev) cudaEventDestroy(e);
    for (int k = 0; k < slots; ++k) ms_out[k] = (k < LBM_NUM_KERNELS && n) ? total[k] / n : 0.0;
    return check_status(h);
}

int lbm_tune(lbm_t *h, int cells_per_thread, int min_blocks_per_sm) {
    if (!h || min_blocks_per_sm < 0) return fail(h, LBM_E_ARG, "lbm_tune: negative min_blocks_per_sm");
    if (h->ready) return fail(h, LBM_E_STATE, "lbm_tune must come before the first step");
    if (cells_per_thread != 0 || min_blocks_per_sm != 0) {
        lbm::Device probe{};
        probe.dom.nx = h->nx;
        probe.precision = h->precision;
        const int v = cells_per_thread ? cells_per_thread : lbm::default_vector_width(probe);
        if (!lbm::valid_variant(probe, v, min_blocks_per_sm))
            return fail(h, LBM_E_ARG, "no bulk kernel with %d cells per thread and %d blocks per SM for nx = %d",
                        v, min_blocks_per_sm, h->nx);
    }
    h->tune_vec = cells_per_thread;
    h->tune_minb = min_blocks_per_sm;
    return LBM_OK;
}

int lbm_debug_set(lbm_t *h, int knob, long long value) {
    if (!h) return LBM_E_ARG;
    if (h->ready && knob != LBM_DEBUG_ADJOINT_SERIAL && knob != LBM_DEBUG_NO_PDL)
        return fail(h, LBM_E_STATE, "lbm_debug_set must come before the first step");
    if (knob == LBM_DEBUG_EXPIRE_WAITS) {
        if (value != 0 && value != 1) return fail(h, LBM_E_ARG, "LBM_DEBUG_EXPIRE_WAITS takes 0 or 1");
        h->expire_waits = (int)value;
    } else if (knob == LBM_DEBUG_CELL_LIST_CAP) {
        if (value < 0) return fail(h, LBM_E_ARG, "LBM_DEBUG_CELL_LIST_CAP takes a capacity >= 1, or 0 for the default");
        h->list_cap_limit = value;
    } else if (knob == LBM_DEBUG_ADJOINT_SERIAL) {
        if (value != 0 && value != 1) return fail(h, LBM_E_ARG, "LBM_DEBUG_ADJOINT_SERIAL takes 0 or 1");
        h->adjoint_sets = value ? 1 : 0;
    } else if (knob == LBM_DEBUG_NO_PDL) {
        if (value != 0 && value != 1) return fail(h, LBM_E_ARG, "LBM_DEBUG_NO_PDL takes 0 or 1");
        if (h->no_pdl != (int)value && h->ready) {
            // the step graphs bake the launch attributes in
            if (int rc = sync_and_check(h)) return rc;
            drop_graphs(h);
        }
        h->no_pdl = (int)value;
    } else {
        return fail(h, LBM_E_ARG, "unknown debug knob %d", knob);
    }
    return LBM_OK;
}

int lbm_autotune(lbm_t *h, int trials, int *best_cells, int *best_blocks) {
    if (!h || trials < 1) return fail(h, LBM_E_ARG, "lbm_autotune: trials must be >= 1");
    int rc = ensure_device(h);
    if (rc) return rc;
    if ((rc = sync_and_check(h))) return rc;
    if (fluid(h)) {
        int vec[64], minb[64];
        const int n = lbm::list_variants(h->dv, vec, minb, 64);
        // time every variant on the buffers of the next step; its populations
        // are rewritten in full by that step, so the state is unchanged
        const lbm::StepPtrs sp = step_ptrs(h, (int)(h->steps & 1));
        cudaEvent_t e0, e1;
        CK(cudaEventCreate(&e0));
        CK(cudaEventCreate(&e1));
        float best = 1e30f;
        int bv = h->dv.vec, bm = h->dv.minb;
        for (int i = 0; i < n; ++i) {
            lbm::Device d = h->dv;
            d.vec = vec[i];
            d.minb = minb[i];
            lbm::launch_stream_collide(d, sp, h->stream);
            CK(cudaEventRecord(e0, h->stream));
            for (int t = 0; t < trials; ++t) lbm::launch_stream_collide(d, sp, h->stream);
            CK(cudaEventRecord(e1, h->stream));
            CK(cudaEventSynchronize(e1));
            float ms = 0;
            CK(cudaEventElapsedTime(&ms, e0, e1));
            if (ms < best) { best = ms; bv = vec[i]; bm = minb[i]; }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        h->dv.vec = h->tune_vec = bv;
        h->dv.minb = h->tune_minb = bm;
        drop_graphs(h);             // the step graphs bake in the launch shape
    }
    if (best_cells) *best_cells = h->dv.vec;
    if (best_blocks) *best_blocks = h->dv.minb;
    return LBM_OK;
}

int lbm_adjoint_record(lbm_t *h, int n, int segment) {
    if (!h || n < 1 || segment < 1)
        return fail(h, LBM_E_ARG, "lbm_adjoint_record: steps and segment must be >= 1");
    if (h->precision != LBM_PREC_F64 && h->precision != LBM_PREC_F32)
        return fail(h, LBM_E_ARG, "the reverse sweep needs FP64 or FP32 storage");
    if (nb(h) == 0) return fail(h, LBM_E_ARG, "the reverse sweep needs at least one body");
    if (h->options & LBM_OPT_AVERAGE_FORCE)
        return fail(h, LBM_E_ARG, "the reverse sweep does not cover LBM_OPT_AVERAGE_FORCE");
    int rc = ensure_device(h);
    if (rc) return rc;
    if ((rc = build_graphs(h))) return rc;
    if ((rc = sync_and_check(h))) return rc;
    auto &tp = h->tape;
    free_list(h, tp.allocs);
    tp.recorded = false;
    const int B = nb(h);
    const long long C = h->C;
    const int nseg = (n + segment - 1) / segment;
    const size_t pop_sz = pop_bytes(h->precision) * lbm::Q * C;
    if ((rc = alloc_list(h, tp.allocs, &tp.state, sizeof(double) * 13 * B * ((size_t)n + 2)))) return rc;
    if ((rc = alloc_list(h, tp.allocs, &tp.force, sizeof(double) * 6 * B * (size_t)n))) return rc;
    if (fluid(h)) {
        if ((rc = alloc_list(h, tp.allocs, &tp.ckpt_pop, pop_sz * nseg))) return rc;
        if ((rc = alloc_list(h, tp.allocs, &tp.ckpt_flags, (size_t)C * nseg))) return rc;
        if ((rc = alloc_list(h, tp.allocs, &tp.ckpt_bid, (size_t)C * nseg))) return rc;
    }
    const long long n0 = h->steps;
    const int p0 = (int)(n0 & 1);
    cudaStream_t s = h->stream;
    const size_t bs = sizeof(BodyState) * B;
    CK(cudaMemcpyAsync(tp.state, h->bodies[p0 ^ 1], bs, cudaMemcpyDeviceToDevice, s));     // state n0 - 1
    CK(cudaMemcpyAsync(tp.state + 13 * B, h->bodies[p0], bs, cudaMemcpyDeviceToDevice, s)); // state n0
    tp.ctl_host = lbm::TapeCtl{tp.state, tp.force, n0, n, 1};
    CK(cudaMemcpyAsync(tp.ctl, &tp.ctl_host, sizeof(lbm::TapeCtl), cudaMemcpyHostToDevice, s));
    for (int k = 0; k < nseg; ++k) {
        const long long m = n0 + (long long)k * segment;
        const int q = (int)((m & 1) ^ 1);           // buffers of epoch m - 1
        if (fluid(h)) {
            CK(cudaMemcpyAsync(static_cast<char *>(tp.ckpt_pop) + pop_sz * k, h->pop[q], pop_sz,
                               cudaMemcpyDeviceToDevice, s));
            CK(cudaMemcpyAsync(tp.ckpt_flags + C * k, h->flags[q], (size_t)C, cudaMemcpyDeviceToDevice, s));
            CK(cudaMemcpyAsync(tp.ckpt_bid + C * k, h->bid[q], (size_t)C, cudaMemcpyDeviceToDevice, s));
        }
        if ((rc = lbm_step(h, std::min(segment, n - k * segment)))) return rc;
    }
    tp.ctl_host.on = 0;
    CK(cudaMemcpyAsync(tp.ctl, &tp.ctl_host, sizeof(lbm::TapeCtl), cudaMemcpyHostToDevice, s));
    if ((rc = sync_and_check(h))) return rc;
    tp.n = n;
    tp.seg = segment;
    tp.nseg = nseg;
    tp.n0 = n0;
    tp.recorded = true;
    return LBM_OK;
}

int lbm_adjoint_backward(lbm_t *h, const double *seed, double *grad_state, double *grad_prev,
                         double *grad_drive, double *grad_spring, double *grad_body, double *grad_pop) {
    if (!h || !seed) return fail(h, LBM_E_ARG, "lbm_adjoint_backward: null seed");
    auto &tp = h->tape;
    if (!tp.recorded) return fail(h, LBM_E_STATE, "lbm_adjoint_backward needs a recording (lbm_adjoint_record)");
    int rc = sync_and_check(h);
    if (rc) return rc;
    // the recomputation remakes the geometry records and the boundary list
    // of the states it replays: the handle's next step prepares its own
    h->need_prep = true;
    const int B = nb(h), ND = (int)h->drives.size(), NS = (int)h->springs.size();
    const long long C = h->C;
    const bool fl = fluid(h);
    const size_t es = pop_bytes(h->precision), as = adj_bytes(h->precision);
    const size_t pop_sz = es * lbm::Q * C;
    const int K = tp.seg;
    std::vector<void *> bk;         // this call's buffers
    // the recomputation's streams (main, side, graph capture) and graphs
    cudaStream_t rs = nullptr, rss = nullptr, rss2 = nullptr, rcap = nullptr, rcaps = nullptr, rcaps2 = nullptr;
    cudaGraphExec_t rgraph[2] = {nullptr, nullptr};
    struct Guard {
        lbm_t *h;
        std::vector<void *> &list;
        cudaStream_t &rs, &rss, &rss2, &rcap, &rcaps, &rcaps2;
        cudaGraphExec_t (&rgraph)[2];
        ~Guard() {
            for (cudaStream_t *st : {&rs, &rss, &rss2, &rcap, &rcaps, &rcaps2})
                if (*st) {
                    cudaStreamSynchronize(*st);
                    cudaStreamDestroy(*st);
                }
            for (cudaGraphExec_t &g : rgraph)
                if (g) cudaGraphExecDestroy(g);
            if (h->side) cudaStreamSynchronize(h->side);
            cudaStreamSynchronize(h->stream);
            free_list(h, list);
        }
    } guard{h, bk, rs, rss, rss2, rcap, rcaps, rcaps2, rgraph};
    // a slot set holds one segment's recomputed epochs: populations (slots
    // 0..K), flags and body ids (slots 0..K+1)
    struct SlotSet {
        void *pop = nullptr;
        uint8_t *flags = nullptr, *bid = nullptr;
    } sets[2];
    uint8_t *carry = nullptr;       // one set: the flags of epoch m + L kept from segment k + 1
    BodyState *stage[2] = {nullptr, nullptr};   // a full segment's states, epochs m - 1 .. m + K - 1
    void *A[2] = {nullptr, nullptr}, *R[2] = {nullptr, nullptr};
    double *sa[2], *fadj, *part, *grads, *r_fh = nullptr, *r_drive_f = nullptr, *r_spring_f = nullptr;
    // the state-only terms of the reversed rigid-body steps of a segment,
    // one set per slot set
    struct TermSet {
        lbm::AdjBodyTerms *tb = nullptr;
        lbm::AdjDriveTerms *td = nullptr;
        lbm::AdjSpringTerms *ts = nullptr;
    } terms[2];
    BodyState *scratch = nullptr;
    lbm::Link *r_links = nullptr;
    int *r_seg = nullptr, *r_changed = nullptr;
    long long *r_t = nullptr;
    const lbm::Device &dv = h->dv;
    const int stride = fl ? lbm::adjoint_part_stride(dv) : 1;
    if ((rc = alloc_list(h, bk, &sa[0], sizeof(double) * 13 * B))) return rc;
    if ((rc = alloc_list(h, bk, &sa[1], sizeof(double) * 13 * B))) return rc;
    if ((rc = alloc_list(h, bk, &fadj, sizeof(double) * 6 * B))) return rc;
    if ((rc = alloc_list(h, bk, &part, sizeof(double) * 9 * B * (size_t)stride))) return rc;
    const size_t ngrad = 2 * (size_t)ND + 3 * (size_t)NS + 5 * (size_t)B;
    if ((rc = alloc_list(h, bk, &grads, sizeof(double) * ngrad))) return rc;
    int nset = 0;
    if (fl) {
        // two sets let segment k - 1 be recomputed while segment k is
        // reversed; the second is taken where the device has ample room
        const size_t set_bytes = pop_sz * (K + 1) + 2 * (size_t)C * (K + 2);
        nset = 1;
        if (h->adjoint_sets != 1 && tp.nseg > 1) {
            size_t free_b = 0, total_b = 0;
            if (cudaMemGetInfo(&free_b, &total_b) == cudaSuccess) {
                if (set_bytes <= total_b / 8 && free_b > 3 * set_bytes) nset = 2;
            } else {
                cudaGetLastError();
            }
        }
        for (int i = 0; i < nset; ++i) {
            if ((rc = alloc_list(h, bk, &stage[i], sizeof(BodyState) * B * (size_t)(K + 1)))) return rc;
            if ((rc = alloc_list(h, bk, &sets[i].pop, pop_sz * (K + 1)))) return rc;
            if ((rc = alloc_list(h, bk, &sets[i].flags, (size_t)C * (K + 2)))) return rc;
            if ((rc = alloc_list(h, bk, &sets[i].bid, (size_t)C * (K + 2)))) return rc;
        }
        if (nset == 1 && (rc = alloc_list(h, bk, &carry, (size_t)C))) return rc;
        for (int i = 0; i < 2; ++i) {
            if ((rc = alloc_list(h, bk, &A[i], as * lbm::Q * C))) return rc;
            if ((rc = alloc_list(h, bk, &R[i], as * C))) return rc;
        }
        if ((rc = alloc_list(h, bk, &scratch, sizeof(BodyState) * B))) return rc;
        if ((rc = alloc_list(h, bk, &r_fh, sizeof(double) * 6 * B))) return rc;
        if ((rc = alloc_list(h, bk, &r_drive_f, sizeof(double) * 3 * std::max(ND, 1)))) return rc;
        if ((rc = alloc_list(h, bk, &r_spring_f, sizeof(double) * 3 * std::max(NS, 1)))) return rc;
        if ((rc = alloc_list(h, bk, &r_links, sizeof(lbm::Link) * (size_t)B * dv.link_side * dv.seg_cap))) return rc;
        if ((rc = alloc_list(h, bk, &r_seg, sizeof(int) * B * dv.link_side))) return rc;
        if ((rc = alloc_list(h, bk, &r_changed, sizeof(int) * 2))) return rc;
        if ((rc = alloc_list(h, bk, &r_t, sizeof(long long)))) return rc;
    }
    for (int i = 0; i < std::max(nset, 1); ++i) {
        if ((rc = alloc_list(h, bk, &terms[i].tb, sizeof(lbm::AdjBodyTerms) * K * std::max(B, 1)))) return rc;
        if ((rc = alloc_list(h, bk, &terms[i].td, sizeof(lbm::AdjDriveTerms) * K * std::max(ND, 1)))) return rc;
        if ((rc = alloc_list(h, bk, &terms[i].ts, sizeof(lbm::AdjSpringTerms) * K * std::max(NS, 1)))) return rc;
    }
    cudaStream_t s = h->stream;
    if ((rc = build_graphs(h))) return rc;        // creates the side stream
    // the bulk part of each reverse step needs no body adjoint: it runs on
    // the side stream, concurrently with the rigid-body and boundary parts;
    // the recomputation runs on a stream of its own
    cudaStream_t side = h->side;
    if (fl) {
        CK(cudaStreamCreateWithFlags(&rs, cudaStreamNonBlocking));
        CK(cudaStreamCreateWithFlags(&rss, cudaStreamNonBlocking));
        CK(cudaStreamCreateWithFlags(&rss2, cudaStreamNonBlocking));
        // the recomputation's graphs run at the greatest priority: its chain
        // bounds the sweep, and the reverse kernels beside it yield SMs
        int least = 0, greatest = 0;
        CK(cudaDeviceGetStreamPriorityRange(&least, &greatest));
        CK(cudaStreamCreateWithPriority(&rcap, cudaStreamNonBlocking, greatest));
        CK(cudaStreamCreateWithPriority(&rcaps, cudaStreamNonBlocking, greatest));
        CK(cudaStreamCreateWithPriority(&rcaps2, cudaStreamNonBlocking, greatest));
    }
    cudaEvent_t ev_main = nullptr, ev_side = nullptr, ev_rec = nullptr, ev_free_main = nullptr,
                ev_free_side = nullptr, ev_rfork = nullptr, ev_rjoin = nullptr, ev_rjoin2 = nullptr, ev_cfork = nullptr,
                ev_cjoin = nullptr, ev_cjoin2 = nullptr;
    CK(cudaEventCreateWithFlags(&ev_main, cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&ev_side, cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&ev_rec, cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&ev_free_main, cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&ev_free_side, cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&ev_rfork, cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&ev_rjoin, cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&ev_cfork, cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&ev_cjoin, cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&ev_rjoin2, cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&ev_cjoin2, cudaEventDisableTiming));
    struct Events {
        cudaEvent_t *e[11];
        ~Events() {
            for (cudaEvent_t *p : e)
                if (*p) cudaEventDestroy(*p);
        }
    } events{{&ev_main, &ev_side, &ev_rec, &ev_free_main, &ev_free_side, &ev_rfork, &ev_rjoin, &ev_cfork, &ev_cjoin,
               &ev_rjoin2, &ev_cjoin2}};
    CK(cudaEventRecord(ev_main, s));
    CK(cudaEventRecord(ev_side, s));
    CK(cudaEventRecord(ev_free_main, s));
    CK(cudaEventRecord(ev_free_side, s));
    double *gd = grads, *gs = grads + 2 * ND, *gb = grads + 2 * ND + 3 * NS;
    CK(cudaMemsetAsync(grads, 0, sizeof(double) * ngrad, s));
    CK(cudaMemsetAsync(part, 0, sizeof(double) * 9 * B * (size_t)stride, s));
    CK(cudaMemcpyAsync(sa[0], seed, sizeof(double) * 13 * B, cudaMemcpyHostToDevice, s));
    int cur = 0;                    // sa[cur]: adjoint of state n + 1
    int ai = 0;                     // A[ai], R[ai]: adjoint entering reverse step n
    // the recomputation runs the forward kernels on its own link lists,
    // change flags, clock, drive and spring forces and force output
    lbm::Device dr = dv;
    dr.hist = nullptr;
    dr.tape = nullptr;
    if (fl) {
        dr.fh = r_fh;
        dr.links = r_links;
        dr.seg_count = r_seg;
        dr.changed = r_changed;
        dr.t_dev = r_t;
        dr.drive_f = r_drive_f;
        dr.spring_f = r_spring_f;
        CK(cudaMemsetAsync(A[0], 0, as * lbm::Q * C, s));
        CK(cudaMemsetAsync(R[0], 0, as * C, s));
        CK(cudaMemsetAsync(r_seg, 0, sizeof(int) * B * dv.link_side, s));
        CK(cudaEventRecord(ev_rec, s));
        CK(cudaStreamWaitEvent(rs, ev_rec, 0));
    }
    const BodyState *states = reinterpret_cast<const BodyState *>(tp.state);
    auto S = [&](long long t) { return states + (t - (tp.n0 - 1)) * B; };     // state t
    auto set_of = [&](int k) -> const SlotSet & { return sets[nset == 2 ? (k & 1) : 0]; };
    auto terms_of = [&](int k) -> const TermSet & { return terms[nset == 2 ? (k & 1) : 0]; };
    // the state-only terms of segment k's steps, on stream st
    auto make_terms = [&](int k, cudaStream_t st) {
        const long long m = tp.n0 + (long long)k * K;
        const TermSet &ts = terms_of(k);
        lbm::launch_adj_terms(dv, S(m), tp.force + (m - tp.n0) * 6 * B, m, std::min(K, tp.n - k * K), ts.tb, ts.td,
                              ts.ts, st);
    };
    auto slot_pop = [&](const SlotSet &st, int j) {
        return static_cast<void *>(static_cast<char *>(st.pop) + pop_sz * j);
    };
    auto seg_len = [&](int k) { return std::min(K, tp.n - k * K); };
    const int ones[2] = {1, 1};
    // recomputation of segment k into its slot set, on rs: epochs m - 1 ..
    // m + L - 1 from the checkpoint (and m + L for the last segment)
    // recomputation step j of a segment into slot set st, the states of
    // epochs j - 1 and j at `prev` and `cur`, on stream `ms` with the side
    // stream `ss`; `last`: only the remap (the flags of the epoch after the
    // run, which the last reverse step needs)
    // The remap rewrites only the cubes around the bodies: a slot starts
    // from the epoch before it, as the forward's ping-pong buffers do.  The
    // copy into slot j + 2 is made after step j's bulk kernel (beside the
    // boundary branch), off the chain; slot 1's before the segment's first
    // remap.  `copy_next`: step j + 1 follows.
    auto copy_slot = [&](const SlotSet &st, int j, cudaStream_t ms) -> int {
        CK(cudaMemcpyAsync(st.flags + C * (j + 1), st.flags + C * j, (size_t)C, cudaMemcpyDeviceToDevice, ms));
        CK(cudaMemcpyAsync(st.bid + C * (j + 1), st.bid + C * j, (size_t)C, cudaMemcpyDeviceToDevice, ms));
        return LBM_OK;
    };
    auto recompute_step = [&](const SlotSet &st, int j, const BodyState *prev, const BodyState *cur, bool last,
                              bool copy_next, cudaStream_t ms, cudaStream_t ss, cudaStream_t ss2,
                              cudaEvent_t fork, cudaEvent_t join, cudaEvent_t join2) -> int {
        int rc3;
        if (j == 0 && (rc3 = copy_slot(st, 0, ms))) return rc3;
        lbm::StepPtrs sp{};
        sp.src = slot_pop(st, j);
        sp.dst = slot_pop(st, j + 1);
        sp.flags_prev = st.flags + C * j;
        sp.bid_prev = st.bid + C * j;
        sp.flags_cur = st.flags + C * (j + 1);
        sp.bid_cur = st.bid + C * (j + 1);
        sp.body_prev = prev;
        sp.body_cur = cur;
        sp.body_next = scratch;
        sp.tstep = dr.t_dev;
        sp.parity = j & 1;
        // the body preparation only at the segment's first step: the later
        // states' geometry records come from the recomputation's own
        // rigid-body steps (the same bits as the tape's states)
        const bool prep = j == 0;
        lbm::launch_remap(dr, sp, 0, ms, prep);
        if (last) return LBM_OK;
        // boundary cells, and link lists with loads, beside the bulk kernel,
        // as in the forward step
        CK(cudaEventRecord(fork, ms));
        CK(cudaStreamWaitEvent(ss, fork, 0));
        if (lbm::needs_boundary_fix(dr)) lbm::launch_boundary_fix(dr, sp, ss);
        CK(cudaEventRecord(join, ss));
        CK(cudaStreamWaitEvent(ss2, fork, 0));
        lbm::launch_links(dr, sp, ss2);
        CK(cudaEventRecord(join2, ss2));
        lbm::launch_stream_collide(dr, sp, ms);
        if (copy_next && (rc3 = copy_slot(st, j + 1, ms))) return rc3;
        CK(cudaStreamWaitEvent(ms, join, 0));
        CK(cudaStreamWaitEvent(ms, join2, 0));
        lbm::launch_force(dr, sp, ms);
        return LBM_OK;
    };
    // A full segment (K steps, not the last) is recomputed by a CUDA graph of
    // its set: its states are staged (epochs m - 1 .. m + K - 1) into the
    // set's staging buffer, so that one graph serves every full segment of
    // the set.
    auto full_graph = [&](int set) -> int {
        if (rgraph[set]) return LBM_OK;
        const SlotSet &st = sets[set];
        CK(cudaStreamBeginCapture(rcap, cudaStreamCaptureModeThreadLocal));
        int rc2 = LBM_OK;
        for (int j = 0; j < K && rc2 == LBM_OK; ++j)
            rc2 = recompute_step(st, j, stage[set] + (long long)j * B, stage[set] + (long long)(j + 1) * B, false,
                                 j + 1 < K, rcap, rcaps, rcaps2, ev_cfork, ev_cjoin, ev_cjoin2);
        cudaGraph_t g = nullptr;
        const cudaError_t e1 = cudaStreamEndCapture(rcap, &g);
        if (rc2) {
            if (g) cudaGraphDestroy(g);
            return rc2;
        }
        CK(e1);
        const cudaError_t e2 = cudaGraphInstantiate(&rgraph[set], g, cudaGraphInstantiateFlagUseNodePriority);
        cudaGraphDestroy(g);
        CK(e2);
        return LBM_OK;
    };
    auto recompute = [&](int k) -> int {
        const long long m = tp.n0 + (long long)k * K;
        const int L = seg_len(k);
        const SlotSet &st = set_of(k);
        const int set = nset == 2 ? (k & 1) : 0;
        if (nset == 1 && k < tp.nseg - 1)       // epoch m + L, recomputed with segment k + 1
            CK(cudaMemcpyAsync(carry, st.flags + C, (size_t)C, cudaMemcpyDeviceToDevice, rs));
        CK(cudaMemcpyAsync(st.pop, static_cast<char *>(tp.ckpt_pop) + pop_sz * k, pop_sz,
                           cudaMemcpyDeviceToDevice, rs));
        CK(cudaMemcpyAsync(st.flags, tp.ckpt_flags + C * k, (size_t)C, cudaMemcpyDeviceToDevice, rs));
        CK(cudaMemcpyAsync(st.bid, tp.ckpt_bid + C * k, (size_t)C, cudaMemcpyDeviceToDevice, rs));
        CK(cudaMemcpyAsync(r_t, &m, sizeof m, cudaMemcpyHostToDevice, rs));
        CK(cudaMemcpyAsync(r_changed, ones, sizeof ones, cudaMemcpyHostToDevice, rs));
        if (L == K && k < tp.nseg - 1) {
            int rc2;
            if ((rc2 = full_graph(set))) return rc2;
            CK(cudaMemcpyAsync(stage[set], S(m - 1), sizeof(BodyState) * B * (size_t)(K + 1),
                               cudaMemcpyDeviceToDevice, rs));
            CK(cudaGraphLaunch(rgraph[set], rs));
        } else {
            const bool extra = k == tp.nseg - 1;    // the remap of the epoch after the run
            for (int j = 0; j < L; ++j) {
                int rc2;
                if ((rc2 = recompute_step(st, j, S(m + j - 1), S(m + j), false, j + 1 < L || extra, rs, rss, rss2,
                                          ev_rfork, ev_rjoin, ev_rjoin2)))
                    return rc2;
            }
            if (extra) {
                int rc2;
                if ((rc2 = recompute_step(st, L, S(m + L - 1), S(m + L), true, false, rs, rss, rss2, ev_rfork, ev_rjoin,
                                          ev_rjoin2)))
                    return rc2;
            }
        }
        make_terms(k, rs);
        CK(cudaGetLastError());
        CK(cudaEventRecord(ev_rec, rs));
        return LBM_OK;
    };
    // segment k's slots are rewritten by the recomputation of segment k - 2
    // (two sets) or k - 1 (one set); it waits for the reverse steps that read
    // them, ev_free_main / ev_free_side (the first reverse step of segment k
    // - 1 reads slot 1 of segment k's set, the flags of epoch m + L, or with
    // one set their copy in carry)
    auto start_recompute = [&](int k) -> int {
        CK(cudaStreamWaitEvent(rs, ev_free_main, 0));
        CK(cudaStreamWaitEvent(rs, ev_free_side, 0));
        return recompute(k);
    };
    if (fl && (rc = start_recompute(tp.nseg - 1))) return rc;
    for (int k = tp.nseg - 1; k >= 0; --k) {
        const long long m = tp.n0 + (long long)k * K;
        const int L = seg_len(k);
        const SlotSet &st = set_of(k);
        if (fl) {
            CK(cudaStreamWaitEvent(s, ev_rec, 0));      // the segment's slots and terms are ready
            CK(cudaEventRecord(ev_main, s));
        } else {
            make_terms(k, s);
        }
        const TermSet &tset = terms_of(k);
        for (int j = L - 1; j >= 0; --j) {
            const long long n = m + j;
            lbm::AdjBody ab{};
            ab.state = S(n);
            ab.fh = tp.force + (n - tp.n0) * 6 * B;
            ab.sa_next = sa[cur];
            ab.sa_cur = sa[cur ^ 1];
            ab.fadj = fadj;
            ab.part = part;
            ab.part_stride = stride;
            ab.part_count = fl ? stride : 0;
            ab.grad_drive = gd;
            ab.grad_spring = gs;
            ab.grad_body = gb;
            ab.tb = tset.tb + (long long)j * B;
            ab.td = tset.td + (long long)j * ND;
            ab.ts = tset.ts + (long long)j * NS;
            ab.t = n;
            lbm::launch_adj_integrate(dv, ab, s);
            if (fl) {
                lbm::AdjPtrs ap{};
                ap.G = slot_pop(st, j + 1);
                ap.flags_cur = st.flags + C * (j + 1);
                ap.bid_cur = st.bid + C * (j + 1);
                ap.bid_prev = st.bid + C * j;
                ap.flags_next = (j + 1 < L || k == tp.nseg - 1) ? st.flags + C * (j + 2)
                                : nset == 2                    ? set_of(k + 1).flags + C
                                                               : carry;
                ap.ain = A[ai];
                ap.rin = R[ai];
                ap.aout = A[ai ^ 1];
                ap.rout = R[ai ^ 1];
                ap.body = S(n);
                ap.fadj = fadj;
                ap.part = part;
                ap.part_stride = stride;
                CK(cudaStreamWaitEvent(side, ev_main, 0));     // Ph^{n+1} of the boundary cells
                lbm::launch_adj_bulk(dv, ap, false, side);
                CK(cudaStreamWaitEvent(s, ev_side, 0));        // Ph^{n+1} of the bulk cells
                CK(cudaEventRecord(ev_side, side));
                lbm::launch_adj_boundary(dv, ap, false, s);
                CK(cudaEventRecord(ev_main, s));
                if (j == L - 1 && nset == 2) {
                    // segment k + 1's set (read up to here) is free for the
                    // recomputation of segment k - 1
                    CK(cudaEventRecord(ev_free_main, s));
                    CK(cudaEventRecord(ev_free_side, side));
                    if (k > 0 && (rc = start_recompute(k - 1))) return rc;
                }
                ai ^= 1;
            }
            cur ^= 1;
        }
        if (fl && nset == 1) {
            CK(cudaEventRecord(ev_free_main, s));
            CK(cudaEventRecord(ev_free_side, side));
            if (k > 0 && (rc = start_recompute(k - 1))) return rc;
        }
        CK(cudaGetLastError());
    }
    // sa[cur]: adjoint of state n0 without the cell sums of reverse step n0
    if (fl) {
        CK(cudaStreamWaitEvent(s, ev_side, 0));
        lbm::launch_adj_reduce(dv, part, stride, stride, sa[cur], s);
        // the stream of step n0 itself: adjoint of the populations entering
        // the run and of the state n0 - 1 (its moving-wall velocities)
        CK(cudaMemsetAsync(fadj, 0, sizeof(double) * 6 * B, s));
        lbm::AdjPtrs ap{};
        ap.G = slot_pop(sets[0], 0);
        ap.flags_cur = sets[0].flags;
        ap.bid_cur = sets[0].bid;
        ap.bid_prev = sets[0].bid;
        ap.flags_next = sets[0].flags + C;
        ap.ain = A[ai];
        ap.rin = R[ai];
        ap.aout = A[ai ^ 1];
        ap.rout = R[ai ^ 1];
        ap.body = S(tp.n0 - 1);
        ap.fadj = fadj;
        ap.part = part;
        ap.part_stride = stride;
        lbm::launch_adj_bulk(dv, ap, true, s);
        lbm::launch_adj_boundary(dv, ap, true, s);
        CK(cudaMemsetAsync(sa[cur ^ 1], 0, sizeof(double) * 13 * B, s));
        lbm::launch_adj_reduce(dv, part, stride, stride, sa[cur ^ 1], s);
        ai ^= 1;
    } else {
        CK(cudaMemsetAsync(sa[cur ^ 1], 0, sizeof(double) * 13 * B, s));
    }
    CK(cudaGetLastError());
    std::vector<double> st(13 * B), pv(13 * B), gh(ngrad);
    CK(cudaMemcpyAsync(st.data(), sa[cur], sizeof(double) * 13 * B, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(pv.data(), sa[cur ^ 1], sizeof(double) * 13 * B, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(gh.data(), grads, sizeof(double) * ngrad, cudaMemcpyDeviceToHost, s));
    if (grad_pop && fl) {
        if (as == 8) {
            CK(cudaMemcpyAsync(grad_pop, A[ai], sizeof(double) * lbm::Q * C, cudaMemcpyDeviceToHost, s));
        } else {
            std::vector<float> tmp((size_t)lbm::Q * C);
            CK(cudaMemcpyAsync(tmp.data(), A[ai], sizeof(float) * lbm::Q * C, cudaMemcpyDeviceToHost, s));
            CK(cudaStreamSynchronize(s));
            for (size_t i = 0; i < tmp.size(); ++i) grad_pop[i] = tmp[i];
        }
    }
    if ((rc = sync_and_check(h))) return rc;
    if (tp.n0 == 0)             // state -1 is state 0: one input
        for (int i = 0; i < 13 * B; ++i) { st[i] += pv[i]; pv[i] = 0.0; }
    if (grad_state) std::memcpy(grad_state, st.data(), sizeof(double) * 13 * B);
    if (grad_prev) std::memcpy(grad_prev, pv.data(), sizeof(double) * 13 * B);
    if (grad_drive)             // device terms are grouped by body: back to creation order
        for (int k = 0; k < ND; ++k)
            for (int i = 0; i < 2; ++i) grad_drive[2 * h->drive_slot[k] + i] = gh[2 * k + i];
    if (grad_spring) std::memcpy(grad_spring, gh.data() + 2 * ND, sizeof(double) * 3 * NS);
    if (grad_body) std::memcpy(grad_body, gh.data() + 2 * ND + 3 * NS, sizeof(double) * 5 * B);
    return LBM_OK;
}

}  // extern "C"

// ---- ensembles ---------------------------------------------------------------

// one storage precision's members of a batched set: the device tables of
// its batched launches (member records, step pointers by parity, and per
// kernel the members' flattened block ranges and grids)
struct EnsGroup {
    int precision = 1;
    int lane = 0;                           // batched mode: the chain of launches the group is in
    std::vector<int> members;               // ensemble indices
    void *mem = nullptr;                    // the tables, one allocation (first member's allocator)
    lbm::Batch bt[lbm::BK_COUNT];           // parity 0 (parity 1 differs only in .parity)
    unsigned blocks[lbm::BK_COUNT] = {};
};

constexpr int ENS_LANES = 2;             // chains of batched launches (see ens_lanes)

struct EnsGraph {
    std::vector<int> set;
    cudaGraphExec_t exec = nullptr;
    std::vector<EnsGroup> groups;           // batched mode only
};

struct lbm_ensemble_s {
    std::vector<lbm_t *> members;
    cudaStream_t stream = nullptr;          // the members' common stream
    cudaStream_t cap = nullptr;             // capture origin
    cudaStream_t side = nullptr;            // batched mode: boundary cells, links and loads beside the bulk kernel
    cudaEvent_t fork = nullptr, bjoin = nullptr;
    // batched mode: the members split into ENS_LANES independent chains of
    // launches, each with its own capture and side streams
    cudaStream_t lcap[ENS_LANES] = {}, lside[ENS_LANES] = {}, lbulk[ENS_LANES] = {};
    cudaEvent_t lfork[ENS_LANES] = {}, ljoin[ENS_LANES] = {}, ldone[ENS_LANES] = {}, lbdone[ENS_LANES] = {};
    cudaEvent_t lstart = nullptr;
    std::vector<cudaEvent_t> join;          // one per member
    int mode = LBM_ENSEMBLE_BATCHED;
    int variant[4] = {-1, -1, -1, -1};      // batched bulk shape per precision (-1: the default)
    // one graph per set of members advanced together (CHUNK_STEPS steps)
    std::vector<EnsGraph> graphs;
    std::vector<unsigned> gens;             // the members' graph generations the cached graphs were built at
    std::string err;
};

namespace {

int ens_fail(lbm_ensemble_t *e, int code, const char *msg) {
    if (e) e->err = msg;
    return code;
}

void ens_drop_graphs(lbm_ensemble_t *e) {
    if (!e->graphs.empty() && e->stream) cudaStreamSynchronize(e->stream);
    for (auto &g : e->graphs) {
        if (g.exec) cudaGraphExecDestroy(g.exec);
        for (auto &grp : g.groups) dfree(e->members[grp.members[0]], grp.mem);
    }
    e->graphs.clear();
}

void ens_release(lbm_ensemble_t *e) {
    ens_drop_graphs(e);
    for (cudaEvent_t ev : e->join) cudaEventDestroy(ev);
    e->join.clear();
    if (e->fork) cudaEventDestroy(e->fork);
    if (e->bjoin) cudaEventDestroy(e->bjoin);
    if (e->cap) cudaStreamDestroy(e->cap);
    if (e->side) cudaStreamDestroy(e->side);
    e->fork = e->bjoin = nullptr;
    e->cap = e->side = nullptr;
    for (int l = 0; l < ENS_LANES; ++l) {
        for (cudaStream_t *st : {&e->lcap[l], &e->lside[l], &e->lbulk[l]})
            if (*st) cudaStreamDestroy(*st);
        for (cudaEvent_t *ev : {&e->lfork[l], &e->ljoin[l], &e->ldone[l], &e->lbdone[l]})
            if (*ev) cudaEventDestroy(*ev);
        e->lcap[l] = e->lside[l] = e->lbulk[l] = nullptr;
        e->lfork[l] = e->ljoin[l] = e->ldone[l] = e->lbdone[l] = nullptr;
    }
    if (e->lstart) cudaEventDestroy(e->lstart);
    e->lstart = nullptr;
}

// can the members of `set` run as batched launches?  (every member has fluid;
// members without bodies skip the body kernels)
bool ens_batchable(const lbm_ensemble_t *e, const std::vector<int> &set) {
    for (int i : set)
        if (!fluid(e->members[i])) return false;
    return true;
}

int ens_variant(const lbm_ensemble_t *e, int precision, const std::vector<int> &members) {
    int v = e->variant[precision];
    auto fits = [&](int var) {
        const int vec = lbm::batch_bulk_shape(precision, var);
        if (vec == 0) return false;
        for (int i : members)
            if (e->members[i]->nx % vec) return false;
        return true;
    };
    if (v >= 0 && fits(v)) return v;
    for (int var : {1, 0})                  // two cells a thread where every nx allows it, else one
        if (fits(var)) return var;
    return 0;
}

// the device tables of one precision group of a batched set
int ens_group_tables(lbm_ensemble_t *e, EnsGroup &g) {
    const int M = (int)g.members.size();
    lbm_t *h0 = e->members[g.members[0]];
    const int variant = ens_variant(e, g.precision, g.members);
    std::vector<lbm::Device> dvs(M);
    std::vector<lbm::StepPtrs> sps(2 * M);
    for (int j = 0; j < M; ++j) {
        lbm_t *h = e->members[g.members[j]];
        dvs[j] = h->dv;
        sps[j] = step_ptrs(h, 0);
        sps[M + j] = step_ptrs(h, 1);
    }
    if (M > 65535) return ens_fail(e, LBM_E_ARG, "more than 65535 members of one precision");
    std::vector<int> tab;                   // per kernel: first[M + 1], grid[3 M]
    std::vector<size_t> off(lbm::BK_COUNT);
    std::vector<unsigned short> owner;      // per kernel, per flattened block: its member
    std::vector<size_t> own_off(lbm::BK_COUNT);
    for (int k = 0; k < lbm::BK_COUNT; ++k) {
        off[k] = tab.size();
        tab.resize(tab.size() + (M + 1) + 3 * M);
        int *first = tab.data() + off[k], *grid = first + M + 1;
        long long total = 0;
        for (int j = 0; j < M; ++j) {
            int gd[3];
            if (k == lbm::BK_BOUNDARY || k == lbm::BK_WALLS || k == lbm::BK_BULK)
                lbm::batch_grid_cells(dvs[j], k, variant, gd);
            else
                lbm::batch_grid_small(dvs[j], k, gd);
            first[j] = (int)total;
            for (int i = 0; i < 3; ++i) grid[3 * j + i] = gd[i];
            total += (long long)gd[0] * gd[1] * gd[2];
        }
        first[M] = (int)total;
        if (total > INT_MAX) return ens_fail(e, LBM_E_ARG, "a batched launch exceeds 2^31 blocks");
        g.blocks[k] = (unsigned)total;
        own_off[k] = owner.size();
        for (int j = 0; j < M; ++j) owner.insert(owner.end(), (size_t)(first[j + 1] - first[j]), (unsigned short)j);
    }
    const size_t b_dv = sizeof(lbm::Device) * M, b_sp = sizeof(lbm::StepPtrs) * 2 * M;
    const size_t o_sp = (b_dv + 255) / 256 * 256, o_tab = o_sp + (b_sp + 255) / 256 * 256;
    const size_t o_own = o_tab + (sizeof(int) * tab.size() + 255) / 256 * 256;
    const size_t bytes = o_own + sizeof(unsigned short) * std::max<size_t>(owner.size(), 1);
    g.mem = dalloc(h0, bytes);
    if (!g.mem) return ens_fail(e, LBM_E_OOM, "device allocation of the ensemble's tables failed");
    char *base = static_cast<char *>(g.mem);
    cudaError_t err = cudaMemcpy(base, dvs.data(), b_dv, cudaMemcpyHostToDevice);
    if (err == cudaSuccess) err = cudaMemcpy(base + o_sp, sps.data(), b_sp, cudaMemcpyHostToDevice);
    if (err == cudaSuccess) err = cudaMemcpy(base + o_tab, tab.data(), sizeof(int) * tab.size(), cudaMemcpyHostToDevice);
    if (err == cudaSuccess && !owner.empty())
        err = cudaMemcpy(base + o_own, owner.data(), sizeof(unsigned short) * owner.size(), cudaMemcpyHostToDevice);
    if (err != cudaSuccess) return ens_fail(e, LBM_E_CUDA, cudaGetErrorString(err));
    const int *dtab = reinterpret_cast<const int *>(base + o_tab);
    for (int k = 0; k < lbm::BK_COUNT; ++k) {
        lbm::Batch &b = g.bt[k];
        b.dv = reinterpret_cast<const lbm::Device *>(base);
        b.sp = reinterpret_cast<const lbm::StepPtrs *>(base + o_sp);
        b.first = dtab + off[k];
        b.grid = dtab + off[k] + M + 1;
        b.member = reinterpret_cast<const unsigned short *>(base + o_own) + own_off[k];
        b.members = M;
        b.parity = 0;
    }
    e->variant[g.precision] = variant;
    return LBM_OK;
}

// one batched step of every group: the kernels of enqueue_step, each as one
// launch over the members of a group
// one batched step of the groups of `lane` on the lane's streams (the bulk
// kernel on `bulk` if not null, else on `main`); `remapped` (if not null) is
// recorded once the step's remap is enqueued
void ens_enqueue_batched(lbm_ensemble_t *e, std::vector<EnsGroup> &groups, int lane, int p, cudaStream_t main,
                         cudaStream_t side, cudaEvent_t fork, cudaEvent_t join, cudaEvent_t remapped,
                         cudaStream_t bulk = nullptr, cudaEvent_t bulk_done = nullptr) {
    auto small = [&](int k, cudaStream_t st) {
        for (auto &g : groups) {
            if (g.lane != lane) continue;
            lbm::Batch b = g.bt[k];
            b.parity = p;
            lbm::launch_batch_small(k, b, g.blocks[k], g.precision, st);
        }
    };
    auto cells = [&](int k, cudaStream_t st) {
        for (auto &g : groups) {
            if (g.lane != lane) continue;
            lbm::Batch b = g.bt[k];
            b.parity = p;
            lbm::launch_batch_cells(k, e->variant[g.precision], b, g.blocks[k], g.precision, st);
        }
    };
    // the batched remap takes its candidates from the body preparation
    small(lbm::BK_PREP, main);
    small(lbm::BK_REMAP, main);
    if (remapped) cudaEventRecord(remapped, main);
    cudaEventRecord(fork, main);
    cudaStreamWaitEvent(side, fork, 0);
    cells(lbm::BK_BOUNDARY, side);
    cells(lbm::BK_WALLS, side);
    small(lbm::BK_LINKS, side);
    small(lbm::BK_LOADS, side);
    cudaEventRecord(join, side);
    if (bulk) {
        cudaStreamWaitEvent(bulk, fork, 0);
        cells(lbm::BK_BULK, bulk);
        cudaEventRecord(bulk_done, bulk);
        cudaStreamWaitEvent(main, bulk_done, 0);
    } else {
        cells(lbm::BK_BULK, main);
    }
    cudaStreamWaitEvent(main, join, 0);
    small(lbm::BK_FORCE, main);
    for (auto &g : groups) {
        if (g.lane != lane) continue;
        for (int i : g.members) {
            lbm_t *h = e->members[i];
            const lbm::StepPtrs sp = step_ptrs(h, p);
            if (nb(h) == 0) lbm::launch_tick(h->dv, sp, main);
            if (h->dv.avg_u) lbm::launch_average(h->dv, sp, main);
        }
    }
}

// Batched sets of two or more members run as ENS_LANES chains of launches
// over halves of the members (balanced by cells).  The second chain starts
// once the first has enqueued its first remap, so while one chain runs its
// latency-bound kernels (prep, remap, force) the other runs its
// bandwidth-bound bulk kernel; the offset persists from step to step.
// Returns the lane of each member of `set` (indexed by ensemble index).
std::vector<int> ens_lanes(const lbm_ensemble_t *e, const std::vector<int> &set) {
    std::vector<int> lane(e->members.size(), 0);
    if (set.size() < 2) return lane;
    std::vector<int> order(set);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return e->members[a]->C > e->members[b]->C; });
    long long load[ENS_LANES] = {};
    for (int i : order) {
        int l = 0;
        for (int k = 1; k < ENS_LANES; ++k)
            if (load[k] < load[l]) l = k;
        lane[i] = l;
        load[l] += e->members[i]->C;
    }
    return lane;
}

// the graph advancing the members `set` by CHUNK_STEPS steps each (built on
// first use).  Batched mode: per step, one launch of each per-step kernel
// over all members of a storage precision.  Branch mode (and sets that
// cannot be batched): fork from the capture origin to every member's
// capture stream, its chunk of steps, join back.
int ens_graph(lbm_ensemble_t *e, const std::vector<int> &set, cudaGraphExec_t *out) {
    for (auto &g : e->graphs)
        if (g.set == set) { *out = g.exec; return LBM_OK; }
    EnsGraph eg;
    eg.set = set;
    const bool batched = e->mode == LBM_ENSEMBLE_BATCHED && ens_batchable(e, set);
    int lanes = 1;
    if (batched) {
        const std::vector<int> lane = ens_lanes(e, set);
        for (int i : set) {
            const int prec = e->members[i]->precision;
            lanes = std::max(lanes, lane[i] + 1);
            EnsGroup *g = nullptr;
            for (auto &x : eg.groups)
                if (x.precision == prec && x.lane == lane[i]) g = &x;
            if (!g) {
                eg.groups.emplace_back();
                g = &eg.groups.back();
                g->precision = prec;
                g->lane = lane[i];
            }
            g->members.push_back(i);
        }
        for (auto &g : eg.groups) {
            const int rc = ens_group_tables(e, g);
            if (rc) {
                for (auto &x : eg.groups)
                    if (x.mem) dfree(e->members[x.members[0]], x.mem);
                return rc;
            }
        }
    }
    cudaGraph_t g = nullptr;
    cudaError_t err = cudaStreamBeginCapture(e->cap, cudaStreamCaptureModeThreadLocal);
    if (err == cudaSuccess) {
        if (batched && lanes == 1) {
            for (int k = 0; k < CHUNK_STEPS; ++k)
                ens_enqueue_batched(e, eg.groups, 0, k & 1, e->cap, e->side, e->fork, e->bjoin, nullptr);
        } else if (batched) {
            cudaEventRecord(e->fork, e->cap);
            for (int l = 0; l < lanes; ++l) cudaStreamWaitEvent(e->lcap[l], e->fork, 0);
            for (int k = 0; k < CHUNK_STEPS; ++k)
                for (int l = 0; l < lanes; ++l) {
                    if (k == 0 && l > 0) cudaStreamWaitEvent(e->lcap[l], e->lstart, 0);
                    ens_enqueue_batched(e, eg.groups, l, k & 1, e->lcap[l], e->lside[l], e->lfork[l], e->ljoin[l],
                                        k == 0 && l + 1 < lanes ? e->lstart : nullptr, e->lbulk[l],
                                        e->lbdone[l]);
                }
            for (int l = 0; l < lanes; ++l) {
                cudaEventRecord(e->ldone[l], e->lcap[l]);
                cudaStreamWaitEvent(e->cap, e->ldone[l], 0);
            }
        } else {
            cudaEventRecord(e->fork, e->cap);
            for (int i : set) {
                lbm_t *h = e->members[i];
                cudaStreamWaitEvent(h->cap, e->fork, 0);
                for (int k = 0; k < CHUNK_STEPS; ++k)
                    enqueue_step(h, k & 1, h->cap, nullptr, nullptr, true, false);
                cudaEventRecord(e->join[i], h->cap);
                cudaStreamWaitEvent(e->cap, e->join[i], 0);
            }
        }
        err = cudaStreamEndCapture(e->cap, &g);
    }
    cudaGraphExec_t x = nullptr;
    if (err == cudaSuccess)
        err = cudaGraphInstantiate(&x, g, batched && lanes > 1 ? cudaGraphInstantiateFlagUseNodePriority : 0);
    if (g) cudaGraphDestroy(g);
    if (err != cudaSuccess) {
        for (auto &grp : eg.groups)
            if (grp.mem) dfree(e->members[grp.members[0]], grp.mem);
        return ens_fail(e, LBM_E_CUDA, cudaGetErrorString(err));
    }
    eg.exec = x;
    e->graphs.push_back(std::move(eg));
    *out = x;
    return LBM_OK;
}

}  // namespace

extern "C" {

int lbm_ensemble_create(lbm_t *const *members, int n, lbm_ensemble_t **out) {
    if (!out) return LBM_E_ARG;
    *out = nullptr;
    if (!members || n < 1) return LBM_E_ARG;
    for (int i = 0; i < n; ++i) {
        if (!members[i]) return LBM_E_ARG;
        for (int j = 0; j < i; ++j)
            if (members[j] == members[i]) return fail(members[i], LBM_E_ARG, "a handle is twice in the ensemble");
        if (members[i]->stream != members[0]->stream)
            return fail(members[i], LBM_E_ARG, "ensemble members must share one stream");
    }
    lbm_ensemble_t *e = new (std::nothrow) lbm_ensemble_s();
    if (!e) return LBM_E_OOM;
    e->members.assign(members, members + n);
    e->stream = members[0]->stream;
    cudaError_t err = cudaStreamCreateWithFlags(&e->cap, cudaStreamNonBlocking);
    if (err == cudaSuccess) err = cudaStreamCreateWithFlags(&e->side, cudaStreamNonBlocking);
    if (err == cudaSuccess) err = cudaEventCreateWithFlags(&e->fork, cudaEventDisableTiming);
    if (err == cudaSuccess) err = cudaEventCreateWithFlags(&e->bjoin, cudaEventDisableTiming);
    // lanes: the latency-bound kernels' streams at the greatest priority,
    // the bulk kernels' at the least, so that one lane's prep, remap and
    // force blocks are dispatched ahead of the other lane's pending bulk blocks
    int least = 0, greatest = 0;
    if (err == cudaSuccess) err = cudaDeviceGetStreamPriorityRange(&least, &greatest);
    for (int l = 0; l < ENS_LANES && err == cudaSuccess; ++l) {
        err = cudaStreamCreateWithPriority(&e->lcap[l], cudaStreamNonBlocking, greatest);
        if (err == cudaSuccess) err = cudaStreamCreateWithPriority(&e->lside[l], cudaStreamNonBlocking, greatest);
        if (err == cudaSuccess) err = cudaStreamCreateWithPriority(&e->lbulk[l], cudaStreamNonBlocking, least);
        for (cudaEvent_t *ev : {&e->lfork[l], &e->ljoin[l], &e->ldone[l], &e->lbdone[l]})
            if (err == cudaSuccess) err = cudaEventCreateWithFlags(ev, cudaEventDisableTiming);
    }
    if (err == cudaSuccess) err = cudaEventCreateWithFlags(&e->lstart, cudaEventDisableTiming);
    for (int i = 0; i < n && err == cudaSuccess; ++i) {
        cudaEvent_t ev = nullptr;
        err = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        if (err == cudaSuccess) e->join.push_back(ev);
    }
    if (err != cudaSuccess) {
        ens_release(e);
        delete e;
        return LBM_E_CUDA;
    }
    *out = e;
    return LBM_OK;
}

int lbm_ensemble_destroy(lbm_ensemble_t *e) {
    if (!e) return LBM_OK;
    if (e->stream) cudaStreamSynchronize(e->stream);
    ens_release(e);
    delete e;
    return LBM_OK;
}

int lbm_ensemble_step(lbm_ensemble_t *e, const int *steps) {
    if (!e || !steps) return ens_fail(e, LBM_E_ARG, "lbm_ensemble_step: null step counts");
    const int n = (int)e->members.size();
    std::vector<long long> left(n);
    for (int i = 0; i < n; ++i) {
        if (steps[i] < 0) return ens_fail(e, LBM_E_ARG, "negative step count");
        left[i] = steps[i];
        lbm_t *h = e->members[i];
        int rc = ensure_device(h);
        if (rc == LBM_OK) rc = build_graphs(h);
        if (rc != LBM_OK) return ens_fail(e, rc, h->err.c_str());
        // members enter a chunk at an even step (the chunk starts with parity 0)
        if (left[i] > 0 && (h->steps & 1)) {
            if ((rc = lbm_step(h, 1))) return ens_fail(e, rc, h->err.c_str());
            --left[i];
        }
    }
    // the members' steps overwrite body buffers that asynchronous reads may
    // still be copying
    for (int i = 0; i < n; ++i) {
        lbm_t *h = e->members[i];
        int rc = wait_read(h, 0);
        if (rc == LBM_OK) rc = wait_read(h, 1);
        if (rc) return ens_fail(e, rc, h->err.c_str());
    }
    // the ensemble's graphs leave the body preparation out: a member whose
    // state the host wrote prepares here
    for (int i = 0; i < n; ++i) {
        lbm_t *h = e->members[i];
        if (left[i] > 0 && h->need_prep && nb(h) > 0 && fluid(h) && !overlapped(h)) {
            lbm::launch_prep(h->dv, step_ptrs(h, (int)(h->steps & 1)), h->stream);
            h->need_prep = false;
        }
    }
    // a member whose step graphs changed (an average begun or stopped, a new
    // launch shape) invalidates the ensemble's graphs
    std::vector<unsigned> gens(n);
    for (int i = 0; i < n; ++i) gens[i] = e->members[i]->graph_gen;
    if (gens != e->gens) {
        ens_drop_graphs(e);
        e->gens = gens;
    }
    for (;;) {
        std::vector<int> set;
        for (int i = 0; i < n; ++i)
            if (left[i] >= CHUNK_STEPS) set.push_back(i);
        if (set.empty()) break;
        cudaGraphExec_t x = nullptr;
        int rc = ens_graph(e, set, &x);
        if (rc) return rc;
        // members whose step budget runs out drop from the set: launch this
        // graph as often as every member of the set has whole chunks left
        long long chunks = left[set[0]] / CHUNK_STEPS;
        for (int i : set) chunks = std::min(chunks, left[i] / CHUNK_STEPS);
        for (long long c = 0; c < chunks; ++c) {
            cudaError_t err = cudaGraphLaunch(x, e->stream);
            if (err != cudaSuccess) return ens_fail(e, LBM_E_CUDA, cudaGetErrorString(err));
        }
        for (int i : set) {
            e->members[i]->steps += chunks * CHUNK_STEPS;
            e->members[i]->tiles_stale = true;      // the ensemble's steps are not overlapped
            left[i] -= chunks * CHUNK_STEPS;
        }
    }
    for (int i = 0; i < n; ++i)
        if (left[i] > 0) {
            int rc = lbm_step(e->members[i], (int)left[i]);
            if (rc) return ens_fail(e, rc, e->members[i]->err.c_str());
        }
    return LBM_OK;
}

int lbm_ensemble_sync(lbm_ensemble_t *e) {
    if (!e) return LBM_E_ARG;
    for (lbm_t *h : e->members) {
        int rc = sync_and_check(h);
        if (rc) return ens_fail(e, rc, h->err.c_str());
    }
    return LBM_OK;
}

const char *lbm_ensemble_last_error(lbm_ensemble_t *e) { return e ? e->err.c_str() : "null handle"; }

int lbm_ensemble_set_mode(lbm_ensemble_t *e, int mode) {
    if (!e || (mode != LBM_ENSEMBLE_BATCHED && mode != LBM_ENSEMBLE_BRANCHES))
        return ens_fail(e, LBM_E_ARG, "lbm_ensemble_set_mode: unknown mode");
    if (mode != e->mode) {
        ens_drop_graphs(e);
        e->mode = mode;
    }
    return LBM_OK;
}

int lbm_ensemble_autotune(lbm_ensemble_t *e, int trials, int *cells_per_thread) {
    if (!e || trials < 1) return ens_fail(e, LBM_E_ARG, "lbm_ensemble_autotune: trials must be >= 1");
    const int n = (int)e->members.size();
    std::vector<int> all(n);
    for (int i = 0; i < n; ++i) {
        all[i] = i;
        lbm_t *h = e->members[i];
        int rc = ensure_device(h);
        if (rc == LBM_OK) rc = sync_and_check(h);
        if (rc) return ens_fail(e, rc, h->err.c_str());
        if ((h->steps & 1) != (e->members[0]->steps & 1))
            return ens_fail(e, LBM_E_STATE, "members must be at steps of the same parity to time the bulk shapes");
    }
    if (!ens_batchable(e, all)) return ens_fail(e, LBM_E_STATE, "a member without fluid cannot be batched");
    const int p = (int)(e->members[0]->steps & 1);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        return ens_fail(e, LBM_E_CUDA, "event creation failed");
    int rc = LBM_OK;
    for (int prec = 0; prec < 4 && rc == LBM_OK; ++prec) {
        EnsGroup g;
        g.precision = prec;
        for (int i = 0; i < n; ++i)
            if (e->members[i]->precision == prec) g.members.push_back(i);
        if (g.members.empty()) continue;
        float best = 1e30f;
        int best_v = -1;
        for (int v = 0; lbm::batch_bulk_shape(prec, v) > 0 && rc == LBM_OK; ++v) {
            bool fits = true;
            for (int i : g.members) fits = fits && e->members[i]->nx % lbm::batch_bulk_shape(prec, v) == 0;
            if (!fits) continue;
            e->variant[prec] = v;
            if ((rc = ens_group_tables(e, g))) break;
            // the populations of every member's next step, which that step rewrites in full
            lbm::Batch b = g.bt[lbm::BK_BULK];
            b.parity = p;
            lbm::launch_batch_cells(lbm::BK_BULK, v, b, g.blocks[lbm::BK_BULK], prec, e->stream);
            cudaEventRecord(e0, e->stream);
            for (int t = 0; t < trials; ++t)
                lbm::launch_batch_cells(lbm::BK_BULK, v, b, g.blocks[lbm::BK_BULK], prec, e->stream);
            cudaEventRecord(e1, e->stream);
            cudaError_t err = cudaEventSynchronize(e1);
            float ms = 0.0f;
            if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
            dfree(e->members[g.members[0]], g.mem);
            g.mem = nullptr;
            if (err != cudaSuccess) { rc = ens_fail(e, LBM_E_CUDA, cudaGetErrorString(err)); break; }
            if (ms < best) { best = ms; best_v = v; }
        }
        e->variant[prec] = best_v;
        if (cells_per_thread && prec == e->members[0]->precision && best_v >= 0)
            *cells_per_thread = lbm::batch_bulk_shape(prec, best_v);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    ens_drop_graphs(e);             // the graphs bake in the bulk shape
    return rc;
}

int lbm_kernels_per_step(lbm_t *h) { return h ? kernels_per_step(h) : LBM_E_ARG; }

int lbm_bytes_per_cell(lbm_t *h) { return h ? (int)(2 * lbm::Q * pop_bytes(h->precision) + 1) : LBM_E_ARG; }

const char *lbm_last_error(lbm_t *h) { return h ? h->err.c_str() : "null handle"; }

}  // extern "C"
#pragma GCC visibility pop
