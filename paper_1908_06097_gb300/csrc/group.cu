// Groups of plans (many truncations and field counts in one call).
#include <vector>

#include "st_internal.cuh"

using namespace st;

struct st_group {
    std::vector<Plan*> plans;
};

extern "C" {

int st_group_create(st_group** out, st_plan* const* plans, int nplans)
{
    if (!out || !plans || nplans < 1 || nplans > 256) {
        set_error("st_group_create: need 1..256 plans");
        return ST_ERR_ARG;
    }
    *out = nullptr;
    st_group* g = new st_group();
    for (int i = 0; i < nplans; i++) {
        if (!plans[i]) {
            delete g;
            set_error("st_group_create: plan %d is NULL", i);
            return ST_ERR_ARG;
        }
        g->plans.push_back((Plan*)plans[i]);
    }
    for (Plan* p : g->plans)
        if (p->opts.prec != g->plans[0]->opts.prec) {
            delete g;
            set_error("st_group_create: plans differ in precision");
            return ST_ERR_ARG;
        }
    *out = g;
    return ST_OK;
}

int st_group_inv(st_group* g, const double* const* spec, double* const* grid, void* stream)
{
    if (!g || !spec || !grid) { set_error("st_group_inv: NULL argument"); return ST_ERR_ARG; }
    for (size_t i = 0; i < g->plans.size(); i++) {
        int rc = st_inv_transform((st_plan*)g->plans[i], spec[i], grid[i], stream);
        if (rc) return rc;
    }
    return ST_OK;
}

int st_group_dir(st_group* g, const double* const* grid, double* const* spec, void* stream)
{
    if (!g || !spec || !grid) { set_error("st_group_dir: NULL argument"); return ST_ERR_ARG; }
    for (size_t i = 0; i < g->plans.size(); i++) {
        int rc = st_dir_transform((st_plan*)g->plans[i], grid[i], spec[i], stream);
        if (rc) return rc;
    }
    return ST_OK;
}

int st_group_destroy(st_group* g)
{
    delete g;
    return ST_OK;
}

}  // extern "C"
