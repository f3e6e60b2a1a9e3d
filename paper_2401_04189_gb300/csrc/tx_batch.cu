// Batched application over many independent systems: one plan, one launch (or one CUDA-graph
// replay) that runs every system's hot path, systems with different contexts concurrently on
// internal streams; plus the autotuner of the expansion tile plan.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <fstream>
#include <map>
#include <sstream>
#include <string>
#include <vector>

#include "tx_internal.h"
#include "tx_tc_ops.h"
#include "tx_paths.h"

namespace tx {
int tc_feasible_plans(const tx_ctx* c, int* bx, int* ns, int cap);
bool tc_current_plan(const tx_ctx* c, int* bx, int* ns);
bool tc_plan_fits(const tx_ctx* c, int bx, int ns);
int tc_describe_plan(const tx_ctx* c, int* out, int nout);
int tc_build_operand_image(tx_ctx* c, cudaStream_t s);
}  // namespace tx

using namespace tx;

struct tx_plan {
    uint32_t magic;
    int device;
    std::vector<tx_batch_item> items;
    std::vector<int> branch;               // internal stream of each item
    std::vector<cudaStream_t> streams;
    std::vector<cudaEvent_t> joins;
    cudaEvent_t fork;
    cudaGraph_t graph;
    cudaGraphExec_t exec;
    std::vector<uint64_t> captured_gen;    // generation of each item's context when the graph was captured
};

static constexpr uint32_t kPlanMagic = 0x54555031u;
static constexpr int kMaxBranches = 8;

static int run_item(const tx_batch_item& it, cudaStream_t s) {
    if (it.e_dev) return tx_exchange_apply_energy(it.ctx, it.psi_occ, it.n_occ, it.out, it.e_dev, (tx_stream_t)s);
    return tx_exchange_apply(it.ctx, it.psi_occ, it.n_occ, it.psi_tgt, it.n_tgt, it.out, (tx_stream_t)s);
}

static std::string shape_key(const tx_ctx* c) {
    std::ostringstream o;
    o << c->n[0] << ' ' << c->n[1] << ' ' << c->n[2] << ' ' << c->r[0] << ' ' << c->r[1] << ' ' << c->r[2] << ' '
      << c->T << ' ' << c->prec;
    return o.str();
}

// tune table: lines "tuxc-tune n1 n2 n3 r1 r2 r3 T prec bx nstage ms"
static std::map<std::string, std::pair<int, int>> read_table(const char* path) {
    std::map<std::string, std::pair<int, int>> t;
    if (!path) return t;
    std::ifstream f(path);
    std::string line;
    while (std::getline(f, line)) {
        std::istringstream in(line);
        std::string tag;
        int v[10];
        double ms;
        if (!(in >> tag) || tag != "tuxc-tune") continue;
        bool okl = true;
        for (int i = 0; i < 10 && okl; ++i) okl = static_cast<bool>(in >> v[i]);
        if (!okl || !(in >> ms)) continue;
        std::ostringstream k;
        k << v[0] << ' ' << v[1] << ' ' << v[2] << ' ' << v[3] << ' ' << v[4] << ' ' << v[5] << ' ' << v[6] << ' '
          << v[7];
        t[k.str()] = {v[8], v[9]};
    }
    return t;
}

static int time_item(const tx_batch_item& it, cudaStream_t s, float* ms) {
    cudaEvent_t a, b;
    TX_TRY_CUDA(cudaEventCreate(&a));
    TX_TRY_CUDA(cudaEventCreate(&b));
    int st = run_item(it, s);   // warm (sizes the workspace, sets attributes)
    if (st == TX_OK) {
        cudaEventRecord(a, s);
        for (int k = 0; k < 2 && st == TX_OK; ++k) st = run_item(it, s);
        cudaEventRecord(b, s);
        cudaEventSynchronize(b);
        cudaEventElapsedTime(ms, a, b);
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return st;
}

static void plan_free(tx_plan* p) {
    if (!p) return;
    if (p->exec) cudaGraphExecDestroy(p->exec);
    if (p->graph) cudaGraphDestroy(p->graph);
    for (auto e : p->joins) cudaEventDestroy(e);
    if (p->fork) cudaEventDestroy(p->fork);
    for (auto s : p->streams) cudaStreamDestroy(s);
    p->magic = 0;
    delete p;
}

extern "C" int tx_set_accumulation_chunk(tx_ctx* c, int terms) {
    if (!c || c->magic != kMagic) return fail(TX_ERR_NOT_SETUP, "context is NULL or was destroyed");
    if (terms < 0) return fail(TX_ERR_INVALID_ARG, "terms must be >= 0");
    c->acc_chunk = terms;
    return TX_OK;
}

extern "C" int tx_set_expansion_form(tx_ctx* c, int form) {
    if (!c || c->magic != kMagic) return fail(TX_ERR_NOT_SETUP, "context is NULL or was destroyed");
    if (form < 0 || form > 5)
        return fail(TX_ERR_INVALID_ARG, "form must be 0 (automatic), 1 (one CTA per item), 2 (bf16 stage 3), 3 "
                                        "(automatic without packed y tiles), 4 (bf16 stage 3 from TMEM) or 5 (dual MMA issuers)");
    if (form == c->consume_form) return TX_OK;
    c->consume_form = form;
    // the two forms' kernels read per-term operator images of different layouts
    if (c->tc && !c->tc->split) return tc_build_operand_image(c, c->last_stream);
    return TX_OK;
}

extern "C" int tx_describe_expansion_plan(const int n[3], const int r[3], int T, int precision, int form, int* out,
                                          int nout) {
    if (!n || !r || !out || nout < 1) return fail(TX_ERR_INVALID_ARG, "n, r and out must not be NULL; nout >= 1");
    if (T < 1) return fail(TX_ERR_INVALID_ARG, "T must be >= 1");
    if (form < 0 || form > 5)
        return fail(TX_ERR_INVALID_ARG, "form must be 0 (automatic), 1 (one CTA per item), 2 (bf16 stage 3), 3 "
                                        "(automatic without packed y tiles), 4 (bf16 stage 3 from TMEM) or 5 (dual MMA issuers)");
    if (precision < TX_PREC_FP32 || precision > TX_PREC_BF16X3)
        return fail(TX_ERR_UNSUPPORTED_PRECISION, "unknown precision");
    for (int d = 0; d < 3; ++d) {
        if (n[d] < 2 || n[d] > 4096) return fail(TX_ERR_SHAPE, "grid sizes must be in [2, 4096]");
        if (r[d] < 1 || r[d] > n[d]) return fail(TX_ERR_SHAPE, "ranks must satisfy 1 <= r_d <= n_d");
    }
    for (int i = 0; i < nout; ++i) out[i] = 0;
    if (precision == TX_PREC_FP32) {
        if (n[2] > 256) return fail(TX_ERR_UNSUPPORTED_SHAPE, "float32 path supports n3 <= 256");
        return TX_OK;
    }
    // a host-side stand-in with the fields the planner reads (no device state)
    tx_ctx c;
    std::memset(&c, 0, sizeof(c));
    for (int d = 0; d < 3; ++d) {
        c.n[d] = n[d];
        c.r[d] = r[d];
    }
    c.T = T;
    c.prec = precision;
    c.consume_form = form;
    std::string why;
    if (!tc_supported(&c, &why)) return fail(TX_ERR_UNSUPPORTED_SHAPE, why);
    return tc_describe_plan(&c, out, nout);
}

extern "C" int tx_set_tile_plan(tx_ctx* c, int bx, int nstage) {
    if (!c || c->magic != kMagic) return fail(TX_ERR_NOT_SETUP, "context is NULL or was destroyed");
    if (bx == 0 && nstage == 0) {
        c->tile_bx = c->tile_nstage = 0;
        return TX_OK;
    }
    if (bx < 1 || nstage < 1 || nstage > 6) return fail(TX_ERR_INVALID_ARG, "bx >= 1 and nstage in 1..6");
    if (c->prec == TX_PREC_FP32) return fail(TX_ERR_UNSUPPORTED_PRECISION, "tile plans apply to tensor-core precisions");
    if (!tc_plan_fits(c, bx, nstage)) return fail(TX_ERR_UNSUPPORTED_SHAPE, "tile plan does not fit SMEM / TMEM");
    c->tile_bx = bx;
    c->tile_nstage = nstage;
    return TX_OK;
}

extern "C" int tx_batch_plan(tx_plan** out, const tx_batch_item* items, int n_items, const char* tune_table,
                             int autotune, tx_stream_t stream) {
    if (!out) return fail(TX_ERR_INVALID_ARG, "plan output pointer is NULL");
    *out = nullptr;
    if (!items || n_items < 1) return fail(TX_ERR_INVALID_ARG, "no items");
    cudaStream_t s = (cudaStream_t)stream;
    for (int i = 0; i < n_items; ++i) {
        const tx_batch_item& it = items[i];
        if (!it.ctx || it.ctx->magic != kMagic) return fail(TX_ERR_NOT_SETUP, "item " + std::to_string(i) + ": bad context");
        if (it.e_dev && it.psi_tgt) return fail(TX_ERR_INVALID_ARG, "item " + std::to_string(i) + ": energy needs psi_tgt == NULL");
        if (!it.psi_occ || !it.out || it.n_occ < 1) return fail(TX_ERR_INVALID_ARG, "item " + std::to_string(i) + ": bad arrays");
    }
    tx_plan* p = new tx_plan();
    p->magic = kPlanMagic;
    p->fork = nullptr;
    p->graph = nullptr;
    p->exec = nullptr;
    cudaGetDevice(&p->device);
    p->items.assign(items, items + n_items);
    // one branch per context (items of a context share its workspace, so they stay in order)
    std::map<const tx_ctx*, int> ctx_branch;
    for (int i = 0; i < n_items; ++i) {
        auto f = ctx_branch.find(items[i].ctx);
        int b;
        if (f == ctx_branch.end()) {
            b = (int)ctx_branch.size() % kMaxBranches;
            ctx_branch[items[i].ctx] = b;
        } else {
            b = f->second;
        }
        p->branch.push_back(b);
    }
    const int nb = std::min<int>(kMaxBranches, (int)ctx_branch.size());
    int st = TX_OK;
    for (int b = 0; b < nb && st == TX_OK; ++b) {
        cudaStream_t ss;
        cudaEvent_t e;
        if (cudaStreamCreateWithFlags(&ss, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess)
            st = fail(TX_ERR_CUDA, "batch streams / events");
        else {
            p->streams.push_back(ss);
            p->joins.push_back(e);
        }
    }
    if (st == TX_OK && cudaEventCreateWithFlags(&p->fork, cudaEventDisableTiming) != cudaSuccess)
        st = fail(TX_ERR_CUDA, "batch fork event");
    // tile plans: table first, then (optionally) autotune the shapes it lacks
    auto table = read_table(tune_table);
    std::map<std::string, bool> done;
    for (int i = 0; i < n_items && st == TX_OK; ++i) {
        tx_ctx* c = items[i].ctx;
        if (c->prec == TX_PREC_FP32) continue;
        const std::string key = shape_key(c);
        if (done.count(key)) {
            // same shape as an earlier item: reuse its decision
            auto t = table.find(key);
            if (t != table.end()) tx_set_tile_plan(c, t->second.first, t->second.second);
            continue;
        }
        done[key] = true;
        auto t = table.find(key);
        if (t != table.end() && tc_plan_fits(c, t->second.first, t->second.second)) {
            tx_set_tile_plan(c, t->second.first, t->second.second);
            continue;
        }
        if (!autotune) continue;
        int bxs[64], nss[64];
        const int nc = tc_feasible_plans(c, bxs, nss, 64);
        float best = 1e30f;
        int bb = 0, bn = 0;
        for (int k = 0; k < nc && st == TX_OK; ++k) {
            tx_set_tile_plan(c, bxs[k], nss[k]);
            float ms = 0.f;
            st = time_item(items[i], s, &ms);
            if (st == TX_OK && ms < best) {
                best = ms;
                bb = bxs[k];
                bn = nss[k];
            }
        }
        if (st != TX_OK) break;
        if (bb > 0) {
            tx_set_tile_plan(c, bb, bn);
            table[key] = {bb, bn};
            if (tune_table) {
                std::ofstream f(tune_table, std::ios::app);
                f << "tuxc-tune " << key << ' ' << bb << ' ' << bn << ' ' << best / 2 << '\n';
            }
        }
    }
    // untimed run of every item: workspaces are sized now, so launches allocate nothing
    for (int i = 0; i < n_items && st == TX_OK; ++i) st = run_item(items[i], s);
    if (st == TX_OK && cudaStreamSynchronize(s) != cudaSuccess) st = fail(TX_ERR_CUDA, "batch warm-up");
    if (st != TX_OK) {
        plan_free(p);
        return st;
    }
    *out = p;
    return TX_OK;
}

extern "C" int tx_batch_launch(tx_plan* p, tx_stream_t stream) {
    if (!p || p->magic != kPlanMagic) return fail(TX_ERR_NOT_SETUP, "plan is NULL or was destroyed");
    for (size_t i = 0; i < p->items.size(); ++i)
        if (ctx_generation(p->items[i].ctx) == 0)
            return fail(TX_ERR_NOT_SETUP, "batch item " + std::to_string(i) + ": its context was destroyed");
    cudaStream_t s = (cudaStream_t)stream;
    TX_TRY_CUDA(cudaEventRecord(p->fork, s));
    for (auto ss : p->streams) TX_TRY_CUDA(cudaStreamWaitEvent(ss, p->fork, 0));
    for (size_t i = 0; i < p->items.size(); ++i) TX_TRY(run_item(p->items[i], p->streams[p->branch[i]]));
    for (size_t b = 0; b < p->streams.size(); ++b) {
        TX_TRY_CUDA(cudaEventRecord(p->joins[b], p->streams[b]));
        TX_TRY_CUDA(cudaStreamWaitEvent(s, p->joins[b], 0));
    }
    return TX_OK;
}

extern "C" int tx_batch_capture(tx_plan* p, tx_stream_t stream) {
    if (!p || p->magic != kPlanMagic) return fail(TX_ERR_NOT_SETUP, "plan is NULL or was destroyed");
    cudaStream_t s = (cudaStream_t)stream;
    if (!s) return fail(TX_ERR_INVALID_ARG, "capture needs a non-default stream");
    if (p->exec) {
        cudaGraphExecDestroy(p->exec);
        p->exec = nullptr;
    }
    if (p->graph) {
        cudaGraphDestroy(p->graph);
        p->graph = nullptr;
    }
    p->captured_gen.clear();
    for (const auto& it : p->items) p->captured_gen.push_back(ctx_generation(it.ctx));
    TX_TRY_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeRelaxed));
    const int st = tx_batch_launch(p, stream);
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(s, &g);
    if (st != TX_OK) {
        if (g) cudaGraphDestroy(g);
        return st;
    }
    // the capture itself must not have replaced a buffer (the plan's warm-up sized them all)
    for (size_t i = 0; i < p->items.size(); ++i)
        if (ctx_generation(p->items[i].ctx) != p->captured_gen[i]) {
            if (g) cudaGraphDestroy(g);
            return fail(TX_ERR_NOT_SETUP, "a context buffer was replaced during capture");
        }
    if (e != cudaSuccess) return fail(TX_ERR_CUDA, std::string("cudaStreamEndCapture: ") + cudaGetErrorString(e));
    p->graph = g;
    TX_TRY_CUDA(cudaGraphInstantiate(&p->exec, g, 0));
    return TX_OK;
}

extern "C" int tx_batch_replay(tx_plan* p, tx_stream_t stream) {
    if (!p || p->magic != kPlanMagic) return fail(TX_ERR_NOT_SETUP, "plan is NULL or was destroyed");
    if (!p->exec) return fail(TX_ERR_NOT_SETUP, "no captured graph (call tx_batch_capture first)");
    // the graph holds raw device pointers of its contexts' workspaces and operand copies:
    // refuse to replay it once any of them was freed, replaced or destroyed
    for (size_t i = 0; i < p->items.size(); ++i) {
        const uint64_t g = ctx_generation(p->items[i].ctx);
        if (g == 0 || i >= p->captured_gen.size() || g != p->captured_gen[i])
            return fail(TX_ERR_NOT_SETUP, "batch item " + std::to_string(i) +
                                              ": its context was destroyed or a buffer it uses was replaced since "
                                              "the capture (call tx_batch_capture again)");
    }
    count_launch();
    TX_TRY_CUDA(cudaGraphLaunch(p->exec, (cudaStream_t)stream));
    return TX_OK;
}

extern "C" int tx_batch_item_plan(const tx_plan* p, int i, int* bx, int* nstage) {
    if (!p || p->magic != kPlanMagic) return fail(TX_ERR_NOT_SETUP, "plan is NULL or was destroyed");
    if (i < 0 || i >= (int)p->items.size() || !bx || !nstage) return fail(TX_ERR_INVALID_ARG, "bad item index");
    *bx = *nstage = 0;
    if (p->items[i].ctx->prec != TX_PREC_FP32) tc_current_plan(p->items[i].ctx, bx, nstage);
    return (int)p->items.size();
}

extern "C" void tx_plan_destroy(tx_plan* p) {
    if (!p || p->magic != kPlanMagic) return;
    cudaDeviceSynchronize();
    plan_free(p);
}
