// Groups of plans: many truncations and field counts, one launch per stage.
//
// A group merges the work lists of its members.  Every work item (a spectral
// chunk, a Legendre tile, a ring-pair transform) carries its member's index,
// and every kernel reads that member's descriptor (tables, workspaces,
// sizes) from a device array built here.  A group transform is therefore six
// kernel launches in total, whatever the number of members:
//   inverse  pre -> Legendre -> ring c2r      direct  ring r2c -> Legendre -> post
// The merged lists are ordered longest first across members (Legendre tiles
// by their contraction length, ring transforms by their FFT length), so the
// short work of small truncations fills in behind the long work of large ones.
// The per-call pointers (each member's spectral and grid arrays) travel by
// value in the launch arguments, so a group call can be captured in a CUDA
// graph like a plan call.
#include <string.h>

#include <algorithm>
#include <vector>

#include "st_internal.cuh"

using namespace st;

struct st_group {
    std::vector<Plan*> plans;
    st_prec prec;
    SpecDesc* d_spec;
    LegDesc *d_leg_inv, *d_leg_dir;
    FftDesc* d_fft;
    int4 *d_spec_work, *d_fft_items, *d_fft_ctas;
    LegTile *d_inv_tiles, *d_dir_tiles;
    int n_spec_work, n_fft_ctas, n_inv_tiles, n_dir_tiles;
    int leg_bn[2];  // Legendre tile widths (inverse, direct) of the group launches
    int last_launches;
    int* d_ctr;     // work counters of the persistent launches of one call (zeroed per call)
};
enum { GROUP_NCTR = 4 };

template <typename X>
static int to_device(X** d, const std::vector<X>& h)
{
    *d = nullptr;
    if (dev_malloc((void**)d, std::max<size_t>(h.size(), 1) * sizeof(X)) != cudaSuccess) {
        cudaGetLastError();
        return ST_ERR_NOMEM;
    }
    if (!h.empty() && cudaMemcpy(*d, h.data(), h.size() * sizeof(X), cudaMemcpyHostToDevice) != cudaSuccess)
        return ST_ERR_CUDA;
    return ST_OK;
}

static void group_free(st_group* g)
{
    if (!g) return;
    void* ptrs[] = {g->d_spec, g->d_leg_inv, g->d_leg_dir, g->d_fft, g->d_spec_work,
                    g->d_fft_items, g->d_fft_ctas, g->d_inv_tiles, g->d_dir_tiles, g->d_ctr};
    for (void* q : ptrs)
        if (q) cudaFree(q);
    delete g;
}

// merged Legendre tile lists for tile widths (bn_inv, bn_dir), longest first
static int group_tiles(st_group* g, int bn_inv, int bn_dir)
{
    std::vector<LegTile> inv, dir;
    for (int i = 0; i < (int)g->plans.size(); i++) {
        std::vector<LegTile> a, b;
        leg_tiles(g->plans[i], 0, bn_inv, bn_dir, a, b);
        for (LegTile& t : a) t.mb = i;
        for (LegTile& t : b) t.mb = i;
        inv.insert(inv.end(), a.begin(), a.end());
        dir.insert(dir.end(), b.begin(), b.end());
    }
    auto kinv = [&](const LegTile& t) { return g->plans[t.mb]->T + 2 - t.m; };
    auto kdir = [&](const LegTile& t) { return g->plans[t.mb]->tab->L[t.m]; };
    std::stable_sort(inv.begin(), inv.end(), [&](const LegTile& a, const LegTile& b) { return kinv(a) > kinv(b); });
    std::stable_sort(dir.begin(), dir.end(), [&](const LegTile& a, const LegTile& b) { return kdir(a) > kdir(b); });
    if (g->d_inv_tiles) cudaFree(g->d_inv_tiles);
    if (g->d_dir_tiles) cudaFree(g->d_dir_tiles);
    g->d_inv_tiles = g->d_dir_tiles = nullptr;
    int rc = to_device(&g->d_inv_tiles, inv);
    if (!rc) rc = to_device(&g->d_dir_tiles, dir);
    g->n_inv_tiles = (int)inv.size();
    g->n_dir_tiles = (int)dir.size();
    g->leg_bn[0] = bn_inv;
    g->leg_bn[1] = bn_dir;
    return rc;
}

static int group_build(st_group* g)
{
    const int n = (int)g->plans.size();
    std::vector<SpecDesc> spec(n);
    std::vector<LegDesc> li(n), ld(n);
    std::vector<FftDesc> fd(n);
    std::vector<int4> swork, items;
    for (int i = 0; i < n; i++) {
        const Plan* p = g->plans[i];
        spec[i] = spec_desc(p);
        li[i] = leg_desc(p, true, p->nfld, p->T);
        ld[i] = leg_desc(p, false, p->nfld, p->T);
        fd[i] = fft_desc(p);
        if (is_split(g->prec) && fd[i].ngop_rows * ((2L * p->nfld + 3) / 4) >= (1L << 31)) {
            set_error("st_group_create: member %d's direct operand is too large for the split kernel", i);
            return ST_ERR_UNSUPPORTED;
        }
        // spectral chunks of 32 degrees x 32 fields
        for (int c = 0; c < p->n_spec_chunks; c++)
            for (int f0 = 0; f0 < p->nfld; f0 += 32) swork.push_back(make_int4(i, c, f0, 0));
        for (int k = 0; k < p->tab->N; k++)
            for (int f = 0; f < p->nfld; f++) items.push_back(make_int4(k, f, i, 0));
    }
    // ring transforms longest first across members
    auto lm = [&](const int4& it) { return g->plans[it.z]->tab->logM[it.x]; };
    std::stable_sort(items.begin(), items.end(), [&](const int4& a, const int4& b) { return lm(a) > lm(b); });
    const std::vector<int4> ctas = fft_ctas(items, lm, fft_cta_points(g->prec));
    int rc = ST_OK;
    if (!rc) rc = to_device(&g->d_spec, spec);
    if (!rc) rc = to_device(&g->d_leg_inv, li);
    if (!rc) rc = to_device(&g->d_leg_dir, ld);
    if (!rc) rc = to_device(&g->d_fft, fd);
    if (!rc) rc = to_device(&g->d_spec_work, swork);
    if (!rc) rc = to_device(&g->d_fft_items, items);
    if (!rc) rc = to_device(&g->d_fft_ctas, ctas);
    g->n_spec_work = (int)swork.size();
    g->n_fft_ctas = (int)ctas.size();
    const int bn0 = leg_bn_candidate(g->prec, 0);
    if (!rc) rc = group_tiles(g, bn0, bn0);
    if (rc) return rc;
    // autotune the tile widths of the merged launches when a member asks for it
    bool tune = false;
    for (const Plan* p : g->plans) tune = tune || (p->opts.flags & ST_FLAG_AUTOTUNE);
    if (!tune) return ST_OK;
    int best_bn[2] = {bn0, bn0};
    for (int dirn = 0; dirn < 2; dirn++) {
        float best = 1e30f;
        for (int v = 0; v < 2; v++) {
            const int bn = leg_bn_candidate(g->prec, v);
            rc = group_tiles(g, bn, bn);
            if (rc) return rc;
            LegArgs A;
            memset(&A, 0, sizeof A);
            A.desc = dirn == 0 ? g->d_leg_inv : g->d_leg_dir;
            A.nmemb = (int)g->plans.size();
            A.tiles = dirn == 0 ? g->d_inv_tiles : g->d_dir_tiles;
            const float ms = time_leg(dirn == 0, g->prec, A, dirn == 0 ? g->n_inv_tiles : g->n_dir_tiles, bn, 3);
            if (ms < 0) return ST_ERR_CUDA;
            if (ms < best) {
                best = ms;
                best_bn[dirn] = bn;
            }
        }
    }
    return group_tiles(g, best_bn[0], best_bn[1]);
}

extern "C" {

int st_group_create(st_group** out, st_plan* const* plans, int nplans)
{
    if (!out || !plans || nplans < 1 || nplans > ST_GROUP_MAX) {
        set_error("st_group_create: need 1..%d plans", (int)ST_GROUP_MAX);
        return ST_ERR_ARG;
    }
    *out = nullptr;
    st_group* g = new st_group();  // value-initialised: every pointer and count is zero
    for (int i = 0; i < nplans; i++) {
        if (!plans[i]) {
            group_free(g);
            set_error("st_group_create: plan %d is NULL", i);
            return ST_ERR_ARG;
        }
        g->plans.push_back((Plan*)plans[i]);
    }
    g->prec = g->plans[0]->opts.prec;
    for (Plan* p : g->plans) {
        if (p->opts.prec != g->prec) {
            group_free(g);
            set_error("st_group_create: plans differ in precision");
            return ST_ERR_ARG;
        }
        if (p->opts.flags & (ST_FLAG_OTF | ST_FLAG_DF64)) {
            group_free(g);
            set_error("st_group_create: plans with ST_FLAG_OTF or ST_FLAG_DF64 cannot be grouped");
            return ST_ERR_UNSUPPORTED;
        }
    }
    int rc = group_build(g);
    if (rc == ST_OK && dev_malloc((void**)&g->d_ctr, GROUP_NCTR * sizeof(int)) != cudaSuccess) rc = ST_ERR_NOMEM;
    if (rc != ST_OK) {
        group_free(g);
        set_error("st_group_create: out of device memory for the merged work lists");
        return rc;
    }
    *out = g;
    return ST_OK;
}

int st_group_inv(st_group* g, const double* const* spec, double* const* grid, void* stream)
{
    if (!g || !spec || !grid) {
        set_error("st_group_inv: NULL argument");
        return ST_ERR_ARG;
    }
    const int n = (int)g->plans.size();
    for (int i = 0; i < n; i++)
        if (!spec[i] || !grid[i]) {
            set_error("st_group_inv: member %d has a NULL array", i);
            return ST_ERR_ARG;
        }
    cudaStream_t s = (cudaStream_t)stream;
    g->last_launches = 0;
    // the spectral and Legendre stages are persistent launches whose CTAs pull
    // the longest-first work list from a counter (the counters restart at 0
    // for each call); the ring FFTs are one plain launch over the merged
    // longest-first CTA list, which the block scheduler hands out in order
    ST_CUDA_TRY(cudaMemsetAsync(g->d_ctr, 0, GROUP_NCTR * sizeof(int), s));
    // pre: spectral operand of every member
    {
        SpecArgs A;
        memset(&A, 0, sizeof A);
        A.desc = g->d_spec;
        A.work = g->d_spec_work;
        A.q = {g->d_ctr + 0, g->n_spec_work};
        A.mode = PRE_PLAIN;
        for (int i = 0; i < n; i++) A.pa[i] = const_cast<double*>(spec[i]);
        int rc = launch_spec(true, g->prec, A, dim3(g->n_spec_work), s);
        if (rc) return rc;
    }
    {
        LegArgs A;
        memset(&A, 0, sizeof A);
        A.desc = g->d_leg_inv;
        A.nmemb = (int)g->plans.size();
        A.tiles = g->d_inv_tiles;
        A.q = {g->d_ctr + 1, g->n_inv_tiles};
        int rc = launch_leg(true, g->prec, A, g->n_inv_tiles, g->leg_bn[0], s);
        if (rc) return rc;
    }
    // FP64: the polar rows of each member in double-double, as st_inv_transform
    int npol = 0;
    for (int i = 0; i < n; i++) {
        Plan* p = g->plans[i];
        if (g->prec != ST_PREC_FP64 || p->tab->npolar <= 0) continue;
        const int keep = p->last_launches;
        int rc = launch_polar(p, PRE_PLAIN, spec[i], nullptr, s);
        p->last_launches = keep;
        if (rc) return rc;
        npol++;
    }
    {
        FftIO io;
        memset(&io, 0, sizeof io);
        io.desc = g->d_fft;
        io.nmemb = (int)g->plans.size();
        io.items = g->d_fft_items;
        io.ctas = g->d_fft_ctas;
        io.narr = 1;
        for (int i = 0; i < n; i++) io.out[i] = grid[i];
        int rc = launch_fft(true, g->prec, io, g->n_fft_ctas, s);
        if (rc) return rc;
    }
    g->last_launches = 3 + npol;  // + the counter reset (a memset, not a kernel)
    return ST_OK;
}

int st_group_dir(st_group* g, const double* const* grid, double* const* spec, void* stream)
{
    if (!g || !spec || !grid) {
        set_error("st_group_dir: NULL argument");
        return ST_ERR_ARG;
    }
    const int n = (int)g->plans.size();
    for (int i = 0; i < n; i++)
        if (!spec[i] || !grid[i]) {
            set_error("st_group_dir: member %d has a NULL array", i);
            return ST_ERR_ARG;
        }
    cudaStream_t s = (cudaStream_t)stream;
    g->last_launches = 0;
    ST_CUDA_TRY(cudaMemsetAsync(g->d_ctr, 0, GROUP_NCTR * sizeof(int), s));
    {
        FftIO io;
        memset(&io, 0, sizeof io);
        io.desc = g->d_fft;
        io.nmemb = (int)g->plans.size();
        io.items = g->d_fft_items;
        io.ctas = g->d_fft_ctas;
        io.narr = 1;
        for (int i = 0; i < n; i++) io.in[i] = grid[i];
        int rc = launch_fft(false, g->prec, io, g->n_fft_ctas, s);
        if (rc) return rc;
        if (is_split(g->prec)) {
            // FP32 operands of the members -> bf16 planes (columns < 2 nfld)
            rc = launch_split_gop(io.d0, g->d_fft, n, 0, s);
            if (rc) return rc;
            g->last_launches++;
        }
    }
    {
        LegArgs A;
        memset(&A, 0, sizeof A);
        A.desc = g->d_leg_dir;
        A.nmemb = (int)g->plans.size();
        A.tiles = g->d_dir_tiles;
        A.q = {g->d_ctr + 1, g->n_dir_tiles};
        int rc = launch_leg(false, g->prec, A, g->n_dir_tiles, g->leg_bn[1], s);
        if (rc) return rc;
    }
    {
        SpecArgs A;
        memset(&A, 0, sizeof A);
        A.desc = g->d_spec;
        A.work = g->d_spec_work;
        A.q = {g->d_ctr + 2, g->n_spec_work};
        A.mode = POST_PLAIN;
        for (int i = 0; i < n; i++) A.pa[i] = spec[i];
        int rc = launch_spec(false, g->prec, A, dim3(g->n_spec_work), s);
        if (rc) return rc;
    }
    g->last_launches += 3;
    return ST_OK;
}

int st_group_destroy(st_group* g)
{
    if (g) cudaDeviceSynchronize();
    group_free(g);
    return ST_OK;
}

int st_group_last_launches(const st_group* g) { return g ? g->last_launches : 0; }

}  // extern "C"
