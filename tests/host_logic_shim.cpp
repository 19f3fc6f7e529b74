// Test shim: the library's CUDA-free host logic behind a C ABI, built with g++ by the CPU tests
// (tests/test_host_layout.py, tests/test_host_noise.py, tests/test_host_forcing.py): the persistent
// kernel's work partition (paper_1703_10119_gb300/csrc/host_layout.h), the noise-table gather
// (csrc/host_noise.h), the fixed-point forcing accumulators (csrc/host_forcing.h) and the host-side fault
// injection (csrc/host_fault.h, tests/test_host_fault.py).
#include "host_fault.h"
#include "host_forcing.h"
#include "host_layout.h"
#include "host_noise.h"

extern "C" {

// out: K, Wl, short_mask, aligned
void shim_wall_layout(int N, const int32_t *first, int nl, int64_t *out)
{
    const hygro::LaneLayout o = hygro::wall_layout(N, first, nl);
    out[0] = o.K;
    out[1] = o.Wl;
    out[2] = (int64_t)o.short_mask;
    out[3] = o.aligned;
}

double shim_sched_cost(int K, int kind)
{
    return hygro::sched_cost({0, K, kind, 0});
}

// Fits the cost model to n walls (K, kind) with measured step times ns; base and out: a[4] then b[4].
int shim_fit_cost_model(int n, const int32_t *K, const int32_t *kind, const double *ns, const double *base, double *out)
{
    std::vector<hygro::SchedWall> w(n);
    std::vector<double> t(ns, ns + n);
    for (int i = 0; i < n; ++i) w[i] = {i, K[i], kind[i], 0};
    hygro::CostModel b, o;
    for (int v = 0; v < 4; ++v) {
        b.a[v] = base[v];
        b.b[v] = base[4 + v];
    }
    const int f = hygro::fit_cost_model(w, t, b, o);
    for (int v = 0; v < 4; ++v) {
        out[v] = o.a[v];
        out[4 + v] = o.b[v];
    }
    return f;
}

// Returns the number of order entries written (at most cap), or -1 when cap is too small.
int shim_lpt_rounds(int n, const int32_t *wall, const int32_t *K, const int32_t *kind, const int32_t *N, int G,
                    int R, int32_t *order, int cap, int32_t *boff, double *load)
{
    std::vector<hygro::SchedWall> w(n);
    for (int i = 0; i < n; ++i) w[i] = {wall[i], K[i], kind[i], N[i]};
    std::vector<int32_t> o, b;
    std::vector<double> l;
    hygro::lpt_rounds(w, G, R, o, b, &l);
    if ((int)o.size() > cap) return -1;
    for (size_t i = 0; i < o.size(); ++i) order[i] = o[i];
    for (int g = 0; g <= G; ++g) boff[g] = b[g];
    for (int g = 0; g < G; ++g) load[g] = l[g];
    return (int)o.size();
}

// n tables of len[k] pairs at src[k] (back to back in the order given); gathers pairs [p0, p1) into dst.
int64_t shim_gather_tables(int n, const float *const *src, const int64_t *len, int64_t p0, int64_t p1, float *dst,
                           int threads, int64_t min_pairs)
{
    std::vector<const float *> s(src, src + n);
    std::vector<int64_t> start(n), l(len, len + n);
    int64_t off = 0;
    for (int k = 0; k < n; ++k) {
        start[k] = off;
        off += l[k];
    }
    return hygro::gather_tables(s, start, l, p0, p1, dst, threads, min_pairs);
}

uint64_t shim_turns_fixed(double x) { return hygro::turns_fixed(x); }

// out: npos0, nstep, n_hi
void shim_noise_fixed(double t0, double dt, double noise_dt, int64_t len, int64_t *out)
{
    const hygro::NoiseFixed o = hygro::noise_fixed(t0, dt, noise_dt, len);
    out[0] = o.npos0;
    out[1] = o.nstep;
    out[2] = o.n_hi;
}

// Parses spec; returns 1 when active (then call_out holds the name, n_out the call to fail), else 0.
int shim_parse_fault(const char *spec, char *call_out, int64_t *n_out)
{
    const hygro::FaultSpec f = hygro::parse_fault(spec);
    if (!f.active) return 0;
    memcpy(call_out, f.call, sizeof f.call);
    *n_out = f.n;
    return 1;
}

// hit_out[i] = 1 when the i-th of the k calls (names[i]) is the one to fail under spec.
void shim_fault_sequence(const char *spec, const char *const *names, int k, int32_t *hit_out)
{
    hygro::FaultInjector inj(hygro::parse_fault(spec));
    for (int i = 0; i < k; ++i) hit_out[i] = inj.hit(names[i]) ? 1 : 0;
}

}  // extern "C"
