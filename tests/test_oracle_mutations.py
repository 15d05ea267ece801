"""Plant plausible mistakes in copies of the oracle source and check that the
pins catch every one of them (CPU only).

Each mutation edits one expression of ``oracle/u1u1_oracle.c`` (a sign, a
factor, an index, a dropped term), the copy is compiled with gcc, and the
pins of ``pins.py`` run against it; at least one must fail.
"""
import os

import pytest

import oracle as O
import pins

MUTATIONS = [
    # name, original text, replacement
    ("current_sign", "(-curl + 2.0 * e2 * c * J)", "(-curl - 2.0 * e2 * c * J)"),
    ("current_factor", "(-curl + 2.0 * e2 * c * J)", "(-curl + e2 * c * J)"),
    ("curl_sign", "(-curl + 2.0 * e2 * c * J)", "(curl + 2.0 * e2 * c * J)"),
    ("backward_link_not_conjugated", "cmul(cconj(link_U(p, st, s, i, xm)), get_phi(p, st, s, xm))",
     "cmul(link_U(p, st, s, i, xm), get_phi(p, st, s, xm))"),
    ("kappa_sign", "0.5 * p->lambda[s] * r_self - p->kappa * r_other",
     "0.5 * p->lambda[s] * r_self + p->kappa * r_other"),
    ("lambda_half", "0.5 * p->lambda[s] * r_self - p->kappa * r_other",
     "p->lambda[s] * r_self - p->kappa * r_other"),
    ("scalar_damping_sign", "((1.0 - delta) * pr + p->deta", "((1.0 + delta) * pr + p->deta"),
    ("omega_definition", "double omega = delta * (1.0 - p->beta);", "double omega = delta * p->beta;"),
    ("coupling_exponent", "double c = pow(a, 2.0 * p->beta);", "double c = pow(a, p->beta);"),
    ("delta_factor", "double delta = 0.5 * p->alpha * pm", "double delta = p->alpha * pm"),
    ("link_convention", "cplx r = {cos(th), -sin(th)};", "cplx r = {cos(th), sin(th)};"),
    ("plaquette_index", "return (get_A(p, st, s, j, xi) - get_A(p, st, s, j, site)",
     "return (get_A(p, st, s, i, xi) - get_A(p, st, s, j, site)"),
    ("curl_neighbour", "long xmj = shift(p, site, j, -1);", "long xmj = shift(p, site, i, -1);"),
    ("link_drift_sign", "st[f_A(s, i) * V + site] += p->deta * v;", "st[f_A(s, i) * V + site] -= p->deta * v;"),
    ("winding_orientation", "- edge_chi(p, st, s, i, xj, &cut) - edge_chi(p, st, s, j, site, &cut);",
     "+ edge_chi(p, st, s, i, xj, &cut) - edge_chi(p, st, s, j, site, &cut);"),
    ("winding_without_links", "tot += p->dx * (get_A(p, st, s, i, site)", "tot += 0.0 * (get_A(p, st, s, i, site)"),
    ("cell_wrong_face", "abs(w[0 * V + site]) + abs(w[0 * V + zp])", "abs(w[0 * V + site]) + abs(w[0 * V + site])"),
    ("overlap_one_sided", "        int hit = 0;\n        for (int dz = -tol; dz <= tol && !hit; ++dz)",
     "        int hit = 0;\n        for (int dz = 0; dz <= tol && !hit; ++dz)"),
    ("kinetic_not_averaged", "kin[s] = 0.5 * (pm2 + pp2);", "kin[s] = pp2;"),
    ("magnetic_factor", "mag[s] = g * f2;", "mag[s] = 0.5 * g * f2;"),
    ("lagrangian_potential_sign", "+ (kin[1] - grad[1] + el[1] - mag[1]) - pot;",
     "+ (kin[1] - grad[1] + el[1] - mag[1]) + pot;"),
    ("gradient_difference", "cplx d = {(fwd.re - f.re) / p->dx, (fwd.im - f.im) / p->dx};",
     "cplx d = {(fwd.re + f.re) / p->dx, (fwd.im + f.im) / p->dx};"),
    ("gauss_charge_factor", "double ct_prev = have_prev ? cfm[5] : 0.0;", "double ct_prev = have_prev ? cfm[2] : 0.0;"),
    ("ic_phase_range", "double th = (2.0 * M_PI) * u;", "double th = M_PI * u;"),
    ("electric_energy_factor", "e2sum += 0.5 * (em * em + ep * ep);", "e2sum += (em * em + ep * ep);"),
    ("components_one_sided", "          for (int dx = -1; dx <= 1; ++dx) {\n            long nb",
     "          for (int dx = 0; dx <= 1; ++dx) {\n            long nb"),
    ("pq_mask_anchor_ignored", "        if (anchor[site] > 0)\n", "        if (anchor[site] >= 0)\n"),
    ("cool_keeps_kappa", "  q.kappa = 0.0;\n", "  q.kappa = p->kappa;\n"),
    ("vint_sign", "double vint = p->kappa * rp * rq;", "double vint = -p->kappa * rp * rq;"),
    ("potential_kappa_sign", "0.25 * p->lambda[1] * rq * rq - p->kappa * rp * rq;",
     "0.25 * p->lambda[1] * rq * rq + p->kappa * rp * rq;"),
    ("self_potential_wrong_sector", "nadd(&acc[D_POT_P], c * 0.25 * p->lambda[0] * rp * rp);",
     "nadd(&acc[D_POT_P], c * 0.25 * p->lambda[1] * rp * rp);"),
    ("cool_step_sign", "st[f_phi(s, c) * V + site] += dt * work", "st[f_phi(s, c) * V + site] -= dt * work"),
    ("scale_factor_inverted", "pow(eta / p->eta_ref, pm)", "pow(p->eta_ref / eta, pm)"),
    ("expansion_exponent", "p->m / (1.0 - p->m)", "p->m / (1.0 + p->m)"),
    ("laplacian_centre_factor", "lap.re += fwd.re + bwd.re - 2.0 * f.re;", "lap.re += fwd.re + bwd.re - 1.0 * f.re;"),
    ("laplacian_dx_power", "double inv_dx2 = 1.0 / (p->dx * p->dx);", "double inv_dx2 = 1.0 / p->dx;"),
    ("scalar_damping_denominator", "((1.0 - delta) * pi + p->deta * (lap.im - g * f.im)) / (1.0 + delta);",
     "((1.0 - delta) * pi + p->deta * (lap.im - g * f.im)) / (1.0 - delta);"),
    ("gauge_damping_denominator", "((1.0 - omega) * Eold + p->deta * (-curl + 2.0 * e2 * c * J)) / (1.0 + omega);",
     "((1.0 - omega) * Eold + p->deta * (-curl + 2.0 * e2 * c * J)) / (1.0 - omega);"),
    ("current_not_over_dx", "double J = t.im / p->dx;", "double J = t.im;"),
    ("curl_not_over_dx", "curl += (plaq_F(p, st, s, i, j, site) - plaq_F(p, st, s, i, j, xmj)) / p->dx;",
     "curl += (plaq_F(p, st, s, i, j, site) - plaq_F(p, st, s, i, j, xmj));"),
    ("phi_drift_sign", "st[f_phi(s, c) * V + site] += p->deta * v;", "st[f_phi(s, c) * V + site] -= p->deta * v;"),
    ("momentum_not_replaced", "st[f_pi(s, c) * V + site] = v;", "st[f_pi(s, c) * V + site] += 0.0 * v;"),
    ("gauge_coupling_not_squared", "double e2 = p->e[s] * p->e[s];", "double e2 = p->e[s];"),
    ("self_coupling_other_sector", "double g = c * (0.5 * p->lambda[s] * r_self",
     "double g = c * (0.5 * p->lambda[o] * r_self"),
    ("current_without_coupling_c", "(-curl + 2.0 * e2 * c * J)", "(-curl + 2.0 * e2 * J)"),
    ("sector_streams_shared", "uint64_t x0 = p->seed ^ ((uint64_t)s << 62);", "uint64_t x0 = p->seed;"),
    ("cut_threshold", "if (M_PI - fabs(chi) < 1e-4 ||", "if (M_PI - fabs(chi) < 1e-1 ||"),
    ("cut_zero_field_ignored", "if (M_PI - fabs(chi) < 1e-4 || (t.re == 0.0 && t.im == 0.0)) *near_cut = 1;",
     "if (M_PI - fabs(chi) < 1e-4) *near_cut = 1;"),
    ("energy_potential_sign", "+ (kin[1] + grad[1] + el[1] + mag[1]) + pot;",
     "+ (kin[1] + grad[1] + el[1] + mag[1]) - pot;"),
    ("energy_magnetic_sign", "double H = (kin[0] + grad[0] + el[0] + mag[0])",
     "double H = (kin[0] + grad[0] + el[0] - mag[0])"),
    ("electric_coupling_factor", "double g = 1.0 / (2.0 * p->e[s] * p->e[s] * c);",
     "double g = 1.0 / (p->e[s] * p->e[s] * c);"),
    ("electric_without_c", "double g = 1.0 / (2.0 * p->e[s] * p->e[s] * c);",
     "double g = 1.0 / (2.0 * p->e[s] * p->e[s]);"),
    ("rl_weight_energy", "nadd(&acc[D_RL_NUM], kt * L);", "nadd(&acc[D_RL_NUM], kt * H);"),
    ("rpq_den_kinetic", "nadd(&acc[D_RPQ_DEN], gt * vint);", "nadd(&acc[D_RPQ_DEN], kt * vint);"),
    ("potential_without_c", "double pot = c * V0;", "double pot = V0;"),
    ("gauss_divergence_forward", "long xm = shift(p, site, i, -1);\n        div +=",
     "long xm = shift(p, site, i, +1);\n        div +="),
    ("phi_extremes_squared", "double mod = sqrt(mod2[s]);", "double mod = mod2[s];"),
    ("charge_sign", "(fr * pi - fi * pr)", "(fi * pr - fr * pi)"),
    ("gradient_conjugate_link", "cplx fwd = cmul(link_U(p, st, s, i, site), get_phi(p, st, s, xp));\n        cplx d",
     "cplx fwd = cmul(cconj(link_U(p, st, s, i, site)), get_phi(p, st, s, xp));\n        cplx d"),
    ("cool_keeps_expansion", "  q.m = 0.0;\n", "  q.m = p->m;\n"),
    ("cool_deta_not_unit", "  q.deta = 1.0;\n", "  q.deta = p->deta;\n"),
    ("cool_keeps_momenta", "    memset(tmp + 10 * V, 0, sizeof(double) * 10 * (size_t)V);\n", "\n"),
    ("cool_links_not_updated", "          st[f_A(s, i) * V + site] += dt * work[4 * V + (3 * s + i) * V + site];",
     "          st[f_A(s, i) * V + site] += 0.0 * work[4 * V + (3 * s + i) * V + site];"),
    ("component_label_neighbour", "              label[nb] = start;", "              label[nb] = c;"),
    ("overlap_anchor_zero_skipped", "        if (anchor[sidx(p, x, y, z)] == 0) continue;",
     "        if (anchor[sidx(p, x, y, z)] > 1) continue;"),
]
# Not listed: keeping the run's beta in the cooling flow (q.beta = p->beta) is
# an equivalent change, since the flow also sets m = 0, so a = 1 and delta = 0
# whatever beta is.


@pytest.mark.parametrize("name,old,new", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_mutation_is_caught(name, old, new, tmp_path):
    src = O.source()
    assert src.count(old) == 1, f"mutation anchor for {name} must occur exactly once"
    lib = O.compile_variant(src.replace(old, new), os.path.join(str(tmp_path), f"lib_{name}.so"))
    caught = []
    with O.use_library(lib):
        for pin in pins.ALL_PINS:
            try:
                pin()
            except Exception as exc:  # noqa: BLE001 - any failure counts as detection
                caught.append((pin.__name__, type(exc).__name__))
                break
    assert caught, f"mutation {name} passed every pin"


# Plausible mistakes in the oracle's host epilogue (oracle/__init__.py: the
# estimators of Eqs. 31-38 formed from the lattice counts, sums and segments).  Each
# mutated copy of the module is executed on its own, and its functions stand
# in for the oracle's while the pins run.
PY_MUTATIONS = [
    ("xi_w_from_p_only", "xi_w=_sqrt_ratio(vol, tot)", "xi_w=_sqrt_ratio(vol, L_p)"),
    ("volume_dx_squared", "    vol = p.nsites * dx ** 3\n    L_pq", "    vol = p.nsites * dx ** 2\n    L_pq"),
    ("f_total_over_p", "f_total=(L_pq / tot)", "f_total=(L_pq / L_p)"),
    ("bound_length_not_removed", "L_p = dx * n_p - L_pq", "L_p = dx * n_p"),
    ("xi_pair_swapped", "xi_p=_sqrt_ratio(vol, L_p), xi_q=_sqrt_ratio(vol, L_q)",
     "xi_p=_sqrt_ratio(vol, L_q), xi_q=_sqrt_ratio(vol, L_p)"),
    ("velocity_factor", "2.0 * R / (1.0 + R)", "R / (1.0 + R)"),
    ("tension_sigma_not_squared", "mu = 2.0 * math.pi * p.sigma[0] ** 2", "mu = 2.0 * math.pi * p.sigma[0]"),
    ("sector_tension_sigma_not_squared", "_sqrt_ratio(-2.0 * math.pi * p.sigma[k] ** 2 * vol, lag_s)",
     "_sqrt_ratio(-2.0 * math.pi * p.sigma[k] * vol, lag_s)"),
    ("segment_length_no_minus_one", "L = p.dx * float((sizes[keep] - 1).sum())", "L = p.dx * float(sizes[keep].sum())"),
    ("segment_threshold_inclusive", "keep = sizes > min_cells", "keep = sizes >= min_cells"),
    ("sector_lag_potential_sign", "- s[\"pot_\" + sec])", "+ s[\"pot_\" + sec])"),
    ("f_p_over_total", "f_p=(L_pq / L_p)", "f_p=(L_pq / tot)"),
    ("v2_pq_from_l_weights", "(\"pq\", \"rpq_num\", \"rpq_den\")", "(\"pq\", \"rl_num\", \"rl_den\")"),
    ("L_pq_without_dx", "L_pq = dx * n_pq_cell", "L_pq = n_pq_cell"),
    ("pq_plaquettes_or", "both = (W[0] != 0) & (W[1] != 0)", "both = (W[0] != 0) | (W[1] != 0)"),
    ("census_w2_strict", "n_w2_p=int((absW[0] >= 2).sum())", "n_w2_p=int((absW[0] > 2).sum())"),
    ("census_cells_strict", "n_cells_ge4_p=int((C[0] >= 4).sum())", "n_cells_ge4_p=int((C[0] > 4).sum())"),
    ("max_w_signed", "max_abs_w=int(absW.max())", "max_abs_w=int(W.max())"),
    ("overlap_q_anchor_same", "n_pq_cell_q = overlap(p, C[1], C[0], tol)", "n_pq_cell_q = overlap(p, C[0], C[1], tol)"),
]


@pytest.mark.parametrize("name,old,new", PY_MUTATIONS, ids=[m[0] for m in PY_MUTATIONS])
def test_epilogue_mutation_is_caught(name, old, new, monkeypatch):
    import sys
    import types
    path = O.__file__
    src = open(path).read()
    assert src.count(old) == 1, f"mutation anchor for {name} must occur exactly once"
    mod = types.ModuleType("oracle_mutant")
    mod.__file__ = path
    mod.__package__ = O.__package__
    monkeypatch.setitem(sys.modules, "oracle_mutant", mod)  # dataclasses look their module up here
    exec(compile(src.replace(old, new), path, "exec"), mod.__dict__)  # noqa: S102 - test of a planted mistake
    mod._lib = O.lib()  # the same compiled oracle
    for fn in ("strings", "diagnostics", "segments"):
        monkeypatch.setattr(O, fn, getattr(mod, fn))
    caught = []
    for pin in pins.ALL_PINS:
        try:
            pin()
        except Exception as exc:  # noqa: BLE001 - any failure counts as detection
            caught.append((pin.__name__, type(exc).__name__))
            break
    assert caught, f"mutation {name} passed every pin"
