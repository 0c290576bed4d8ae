// Body sets of an iFCI system and their frozen-body orbital lists (host side),
// shared by ifci_increments and ifci_rdm_backward.
#pragma once
#include <algorithm>
#include <cmath>
#include <map>

#include "common.cuh"

namespace ifci {

// All body sets of size 1..max_order: by size, then lexicographic.
inline void enumerate_subsets(int nbody, int max_order, std::vector<std::vector<int>> &out) {
    out.clear();
    for (int k = 1; k <= max_order; k++) {
        std::vector<int> c(k);
        for (int i = 0; i < k; i++) c[i] = i;
        while (true) {
            out.push_back(c);
            int i = k - 1;
            while (i >= 0 && c[i] == nbody - k + i) i--;
            if (i < 0) break;
            c[i]++;
            for (int j = i + 1; j < k; j++) c[j] = c[j - 1] + 1;
        }
    }
}

struct SystemView {
    const double *h = nullptr, *V = nullptr;   // device
};

inline int validate_system(ifci_handle_t h, const ifci_system_t *sys, int max_order) {
    if (!sys || !sys->body_offset || !sys->h || !sys->eri || sys->nbody < 1)
        return set_error(h, IFCI_ERR_INVALID_ARG, "system: null field");
    if (max_order < 1 || max_order > sys->nbody)
        return set_error(h, IFCI_ERR_INVALID_ARG, "system: max_order %d with %d bodies", max_order, sys->nbody);
    if (sys->body_offset[0] != 0 || sys->body_offset[sys->nbody] != sys->norb)
        return set_error(h, IFCI_ERR_INVALID_ARG, "system: body_offset must run from 0 to norb");
    for (int b = 0; b < sys->nbody; b++)
        if (sys->body_offset[b + 1] <= sys->body_offset[b])
            return set_error(h, IFCI_ERR_INVALID_ARG, "system: body %d has no orbitals", b);
    return IFCI_OK;
}

struct SubsetPlan {
    std::vector<std::vector<int>> subsets;
    std::vector<int> nA, nC;
    std::vector<int> orbs;          // per subset: active..., core...
    std::vector<long long> orb_off;
    std::vector<long long> sub_off;
    std::vector<int> sub_idx;
    std::vector<signed char> sub_sgn;
};

inline void plan_subsets(const ifci_system_t *sys, int max_order, SubsetPlan &P) {
    enumerate_subsets(sys->nbody, max_order, P.subsets);
    const int ns = (int)P.subsets.size();
    // position lookup of a subset: per size, lexicographic rank
    std::vector<long long> size_off(max_order + 2, 0);
    for (int k = 1; k <= max_order; k++) size_off[k + 1] = size_off[k] + binom(sys->nbody, k);
    auto rank_of = [&](const std::vector<int> &Y) -> long long {
        // lexicographic rank among |Y|-subsets of nbody
        int k = (int)Y.size(), N = sys->nbody;
        long long r = 0;
        int prev = -1;
        for (int i = 0; i < k; i++) {
            for (int v = prev + 1; v < Y[i]; v++) r += binom(N - 1 - v, k - 1 - i);
            prev = Y[i];
        }
        return size_off[k] + r;
    };
    P.sub_off.assign(1, 0);
    for (int x = 0; x < ns; x++) {
        const std::vector<int> &X = P.subsets[x];
        const int k = (int)X.size();
        std::vector<char> in(sys->nbody, 0);
        for (int b : X) in[b] = 1;
        P.orb_off.push_back((long long)P.orbs.size());
        int na = 0;
        for (int b = 0; b < sys->nbody; b++)
            if (in[b])
                for (int p = sys->body_offset[b]; p < sys->body_offset[b + 1]; p++, na++) P.orbs.push_back(p);
        int nc = 0;
        for (int b = 0; b < sys->nbody; b++)
            if (!in[b]) { P.orbs.push_back(sys->body_offset[b]); nc++; }
        P.nA.push_back(na);
        P.nC.push_back(nc);
        for (int mask = 1; mask < (1 << k); mask++) {
            std::vector<int> Y;
            for (int i = 0; i < k; i++)
                if (mask >> i & 1) Y.push_back(X[i]);
            P.sub_idx.push_back((int)rank_of(Y));
            P.sub_sgn.push_back(((k - (int)Y.size()) & 1) ? -1 : 1);
        }
        P.sub_off.push_back((long long)P.sub_idx.size());
    }
}


// Position of the pair {a, b} (a < b) in the subset order (all single bodies first).
inline long long pair_position(int nbody, int a, int b) {
    return nbody + (long long)a * nbody - (long long)a * (a + 1) / 2 + (b - a - 1);
}

// Connected n-body screening: the bodies of X, joined by the pairs of X with
// |eps_pair| >= C, form one connected graph.
inline bool cnb_connected(const std::vector<int> &X, int nbody, const std::vector<double> &eps, double C) {
    const int k = (int)X.size();
    std::vector<char> seen(k, 0);
    std::vector<int> stack{0};
    seen[0] = 1;
    int nseen = 1;
    while (!stack.empty()) {
        const int i = stack.back();
        stack.pop_back();
        for (int j = 0; j < k; j++) {
            if (seen[j]) continue;
            const int a = std::min(X[i], X[j]), b = std::max(X[i], X[j]);
            if (std::fabs(eps[pair_position(nbody, a, b)]) >= C) {
                seen[j] = 1;
                nseen++;
                stack.push_back(j);
            }
        }
    }
    return nseen == k;
}

// d(sum_X eps_X) / d E_c(Y) for the recursion of Eqs. 2-5 with screened sets
// (included[x] = 0) counting as zero: eps_X = E_c(X) - sum_{Y proper subset} eps_Y.
// The coefficients of eps_X over the E_c of its subsets follow the same
// recursion; the weights are their sums over the included sets.
inline std::vector<double> screened_weights(const SubsetPlan &P, const std::vector<char> &included) {
    const int ns = (int)P.subsets.size();
    std::vector<std::vector<std::pair<int, double>>> coef(ns);
    std::vector<double> w(ns, 0.0);
    for (int x = 0; x < ns; x++) {
        if (!included[x]) continue;
        std::map<int, double> cx;
        cx[x] += 1.0;
        for (long long t = P.sub_off[x]; t < P.sub_off[x + 1]; t++) {
            const int y = P.sub_idx[t];
            if (y == x || !included[y]) continue;
            for (const auto &e : coef[y]) cx[e.first] -= e.second;
        }
        coef[x].assign(cx.begin(), cx.end());
        for (const auto &e : coef[x]) w[e.first] += e.second;
    }
    return w;
}

}  // namespace ifci
