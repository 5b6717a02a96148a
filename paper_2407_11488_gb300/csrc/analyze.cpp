// Analysis of a timing table: the tuning-impact statistics of Sec. 4 and the
// proportion of centrality of Eq. 1 on the fitness flow graph.
//
// Fitness flow graph: one node per measured configuration; an edge x -> y
// when y is a neighbour of x (one parameter moved one step in its ordered
// value list) and y is strictly faster.  Centrality is PageRank (damping
// 0.85, uniform teleport, a sink's mass spread uniformly).  Local minima are
// the sinks.  C_p = centrality of the minima within (1+p) of the optimum
// (inclusive) / centrality of all minima.
#include "ct_internal.hpp"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <unordered_map>

using namespace ct;

namespace {

// numpy's default percentile: linear interpolation between order statistics
double percentile(const std::vector<double>& sorted, double q)
{
    if (sorted.empty()) return NAN;
    const double pos = q / 100.0 * (double)(sorted.size() - 1);
    const size_t lo = (size_t)std::floor(pos), hi = (size_t)std::ceil(pos);
    const double f = pos - (double)lo;
    return sorted[lo] + (sorted[hi] - sorted[lo]) * f;
}

double median(std::vector<double> v)
{
    std::sort(v.begin(), v.end());
    const size_t n = v.size();
    if (!n) return NAN;
    return n % 2 ? v[n / 2] : 0.5 * (v[n / 2 - 1] + v[n / 2]);
}

}  // namespace

extern "C" CT_API ct_status ct_table_analyze(const ct_table* t, const ct_space* s, double flops, const double* p_values,
                                             int32_t n_p, ct_analysis* out)
{
    if (!t || !s || !out) return fail(CT_ERR_INVALID_ARG, "table, space and out must be non-NULL");
    if (n_p < 0 || n_p > 16 || (n_p > 0 && !p_values)) return fail(CT_ERR_INVALID_ARG, "0..16 p values");
    memset(out, 0, sizeof *out);
    // nodes: measured configurations
    std::vector<const ct_row*> nodes;
    for (const auto& r : t->rows)
        if (r.status == CT_OK && std::isfinite(r.t_med_ms) && r.t_med_ms > 0) nodes.push_back(&r);
    if (nodes.empty()) return fail(CT_ERR_INVALID_ARG, "the table has no measured configuration");
    const size_t n = nodes.size();
    std::vector<double> tm(n), perf(n);
    size_t best = 0;
    for (size_t i = 0; i < n; ++i) {
        tm[i] = nodes[i]->t_med_ms;
        perf[i] = flops > 0 ? flops / (tm[i] * 1e-3) / 1e9 : 1.0 / tm[i];
        if (tm[i] < tm[best] || (tm[i] == tm[best] && nodes[i]->index < nodes[best]->index)) best = i;
    }
    const double t_opt = tm[best];
    out->n_valid = (int64_t)n;
    out->best_index = nodes[best]->index;
    out->p_max = perf[best];
    out->p_median = median(perf);
    out->impact = out->p_max / out->p_median;
    out->tuned_vs_median = median(tm) / t_opt;
    size_t within = 0;
    for (double x : tm) within += x <= 1.10 * t_opt ? 1 : 0;
    out->frac_within_10pct = (double)within / (double)n;
    std::vector<double> ps = perf;
    std::sort(ps.begin(), ps.end());
    const double qs[7] = {0, 10, 25, 50, 75, 90, 100};
    for (int k = 0; k < 7; ++k) out->quantiles[k] = percentile(ps, qs[k]);

    // fitness flow graph over the measured configurations
    std::unordered_map<int64_t, size_t> pos;
    for (size_t i = 0; i < n; ++i) pos[nodes[i]->index] = i;
    std::vector<std::vector<size_t>> edges(n);
    for (size_t i = 0; i < n; ++i) {
        const ct_config& c = nodes[i]->cfg;
        for (int k = 0; k < 6; ++k) {
            const auto& vals = s->s.vals[k];
            int p = -1;
            for (size_t j = 0; j < vals.size(); ++j)
                if (vals[j] == cfg_get(c, k)) p = (int)j;
            if (p < 0) return fail(CT_ERR_INVALID_ARG, "table row outside the space");
            for (int d : {-1, 1}) {
                const int q = p + d;
                if (q < 0 || q >= (int)vals.size()) continue;
                ct_config nb = c;
                cfg_set(nb, k, vals[q]);
                const int64_t idx = s->s.index_of(nb);
                auto it = pos.find(idx);
                if (it != pos.end() && tm[it->second] < tm[i]) edges[i].push_back(it->second);
            }
        }
    }
    // PageRank by power iteration
    const double d = 0.85;
    std::vector<double> r(n, 1.0 / (double)n), nx(n);
    for (int it = 0; it < 100000; ++it) {
        double sink = 0.0;
        std::fill(nx.begin(), nx.end(), (1.0 - d) / (double)n);
        for (size_t i = 0; i < n; ++i) {
            if (edges[i].empty()) {
                sink += r[i];
            } else {
                const double share = d * r[i] / (double)edges[i].size();
                for (size_t j : edges[i]) nx[j] += share;
            }
        }
        double diff = 0.0;
        for (size_t i = 0; i < n; ++i) {
            nx[i] += d * sink / (double)n;
            diff += std::fabs(nx[i] - r[i]);
        }
        r.swap(nx);
        if (diff < 1e-13) break;
    }
    double den = 0.0;
    int64_t minima = 0;
    for (size_t i = 0; i < n; ++i)
        if (edges[i].empty()) {
            den += r[i];
            minima++;
        }
    out->n_minima = minima;
    out->n_p = n_p;
    for (int k = 0; k < n_p; ++k) {
        double num = 0.0;
        for (size_t i = 0; i < n; ++i)
            if (edges[i].empty() && tm[i] <= (1.0 + p_values[k]) * t_opt) num += r[i];
        out->p[k] = p_values[k];
        out->cp[k] = den > 0 ? num / den : NAN;
    }
    return CT_OK;
}
