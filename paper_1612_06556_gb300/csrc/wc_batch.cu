// Batched solves over several lattices / right-hand sides.
#include "wc_internal.cuh"

namespace wc {
wc_status bicgstab(wc_lattice lat, int kind, wc_field x, wc_field b, const wc_solve_params &p, wc_solve_info *info);
wc_status check_solve_args(wc_lattice lat, wc_field x, wc_field b, const wc_solve_params *p);
}  // namespace wc

using namespace wc;

extern "C" wc_status wc_solve_batch(int n, const wc_lattice *lats, wc_field *xs, wc_field *bs,
                                    const wc_solve_params *p, wc_solve_info *infos)
{
    if (n < 0 || (n > 0 && (!lats || !xs || !bs || !p || !infos)))
        return set_error(nullptr, WC_ERR_ARG, "wc_solve_batch: bad arguments");
    for (int i = 0; i < n; ++i) {
        wc_status st = check_solve_args(lats[i], xs[i], bs[i], p);
        if (st != WC_OK) return st;
    }
    wc_status worst = WC_OK;
    for (int i = 0; i < n; ++i) {
        wc_status st = bicgstab(lats[i], 0, xs[i], bs[i], *p, &infos[i]);
        if (st != WC_OK && worst == WC_OK) worst = st;
    }
    return worst;
}
