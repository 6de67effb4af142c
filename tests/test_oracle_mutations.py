"""The oracle's pins are strong enough to catch plausible mistakes.

Each case plants one mistake in a temporary copy of the oracle's C source (a
dropped term, a wrong sign, coefficient or index, a swapped operand), builds
it, and runs the oracle pin suites against that build in a subprocess: at
least one pin must fail.  Nothing here touches the real oracle build.
"""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "mfc5_oracle.c")
MLP_SRC = os.path.join(ROOT, "oracle", "mlp_oracle.c")

MUTATIONS = {
    "drop_alpha_source": ("L[IA(g) + k] = L[IA(g) + k] + ak * (UF[i + 1] - UF[i]) / dx;", "L[IA(g) + k] = L[IA(g) + k];"),
    "source_sign": ("L[IA(g) + k] = L[IA(g) + k] + ak * (UF[i + 1] - UF[i]) / dx;",
                    "L[IA(g) + k] = L[IA(g) + k] - ak * (UF[i + 1] - UF[i]) / dx;"),
    "alpha_flux_uK": ("F[IA(g) + i] = K->a[i] * Ss;", "F[IA(g) + i] = K->a[i] * un;"),
    "beta0_coefficient": ("0.25 * sq(v[0] - 4.0 * v[1] + 3.0 * v[2])", "0.25 * sq(v[0] - 4.0 * v[1] + 2.0 * v[2])"),
    "linear_weight": ("double a0 = 0.1 / sq(eps + b0);", "double a0 = 0.3 / sq(eps + b0);"),
    "candidate_index": ("double p1 = (-v[1] + 5.0 * v[2] + 2.0 * v[3]) / 6.0;",
                        "double p1 = (-v[1] + 5.0 * v[2] + 2.0 * v[4]) / 6.0;"),
    "eps_power": ("double a1 = 0.6 / sq(eps + b1);", "double a1 = 0.6 / (eps + b1);"),
    "face_states_swapped": ("hllc(g, d, &VM[(j + 1) * neq], &VP[(j + 2) * neq]",
                            "hllc(g, d, &VP[(j + 1) * neq], &VM[(j + 2) * neq]"),
    "star_energy_sign": ("(Ss - un) * (K->rho * Ss + K->p / (SK - un))",
                         "(Ss - un) * (K->rho * Ss - K->p / (SK - un))"),
    "star_tangential": ("chi * K->rho * K->u[k];", "K->rho * K->u[k];"),
    "chi_shifted": ("double chi = (SK - un) / (SK - Ss);", "double chi = (SK - un) / (SK - Ss + 1e-3);"),
    "sstar_sign": ("double num = R.p - L.p + L.rho", "double num = L.p - R.p + L.rho"),
    "davis_right": ("double SR = (uL + cL > uR + cR) ? uL + cL : uR + cR;", "double SR = uR + cR;"),
    "face_velocity": ("        star_flux(g, dir, wL, &L, SL, Ss, F);\n        *uf = Ss;",
                      "        star_flux(g, dir, wL, &L, SL, Ss, F);\n        *uf = uL;"),
    "momentum_pressure": ("F[IU(g) + dir] = F[IU(g) + dir] + K->p;", "F[IU(g) + dir] = F[IU(g) + dir];"),
    "energy_flux": ("F[IE(g)] = (K->E + K->p) * un;", "F[IE(g)] = (K->E) * un;"),
    "sound_speed": ("return ((G + 1.0) * p + Pi) / (G * rho);", "return ((G + 1.0) * p + Pi) / (rho);"),
    "mixture_Pi": ("*Pi = sp + aN * g->Pk[g->nf - 1];", "*Pi = sp + a[0] * g->Pk[g->nf - 1];"),
    "mixture_Gamma": ("*G = sg + aN * g->gk[g->nf - 1];", "*G = sg + aN * g->gk[0];"),
    "kinetic_half": ("return 0.5 * rho * s;", "return rho * s;"),
    "rk_stage2": ("0.75 * q[i] + 0.25 * (q1[i] + dt * L[i])", "0.75 * q[i] + 0.25 * (q1[i] + 0.5 * dt * L[i])"),
    "rk_stage3": ("(2.0 / 3.0) * (q2[i] + dt * L[i])", "(2.0 / 3.0) * (q2[i] + dt * L[i] * 0.99)"),
    "periodic_ghosts": ("if (periodic) {", "if (0) {"),
    "wavespeed_dx": ("(fabs(w[IU(&g) + d]) + cs) / cell_width(&g, d, (c / g.stride[d]) % g.n[d]);",
                     "(fabs(w[IU(&g) + d]) + cs);"),
    "weno3_linear_weight": ("double a0 = (1.0 / 3.0) / sq(eps + b0);", "double a0 = (2.0 / 3.0) / sq(eps + b0);"),
    "weno3_candidate_index": ("double p1 = (v[2] + v[3]) / 2.0;", "double p1 = (v[2] + v[4]) / 2.0;"),
    "weno3_beta_index": ("double b1 = sq(v[3] - v[2]);", "double b1 = sq(v[3] - v[1]);"),
    "weno3_right_candidate": ("p1 = (3.0 * v[2] - v[3]) / 2.0;", "p1 = (3.0 * v[2] + v[3]) / 2.0;"),
    "weno_order_ignored": ("    if (g->order == 3)\n        weno3(", "    if (0)\n        weno3("),
    "nu_beta_coefficient": ("beta[k] = b * b + (13.0 / 3.0) * (c * c);", "beta[k] = b * b + (13.0 / 12.0) * (c * c);"),
    "nu_linear_weight": ("dp[2] = Qp[4] / cp[3 * 2 + 2];", "dp[2] = Qp[4] / cp[3 * 2 + 1];"),
    "nu_face_value": ("cp[3 * k + j] = Mi[j] + 0.5 * Mi[3 + j] + 0.25 * Mi[6 + j];",
                      "cp[3 * k + j] = Mi[j] + 0.5 * Mi[3 + j] + 0.5 * Mi[6 + j];"),
    "nu_global_width": ("double dx = cell_width(g, d, i);", "double dx = g->dx[d];"),
    "nf_mixture_middle": ("sg = sg + a[i] * g->gk[i];", "sg = sg + a[i] * g->gk[0];"),
    "nf_source_loop": ("for (int k = 0; k < g->nf - 1; k++) {\n                    double ak",
                       "for (int k = 0; k < 1; k++) {\n                    double ak"),
    "nf_star_density": ("for (int i = 0; i < g->nf; i++) F[i] = F[i] + SK * (chi * w[i] - w[i]);",
                        "for (int i = 0; i < 2; i++) F[i] = F[i] + SK * (chi * w[i] - w[i]);"),
    "nf_rho": ("for (int i = 2; i < g->nf; i++) rho = rho + q[i];", "for (int i = 3; i < g->nf; i++) rho = rho + q[i];"),
    "nf_alpha_flux": ("for (int i = 0; i < g->nf - 1; i++) F[IA(g) + i] = K->a[i] * un;",
                      "for (int i = 0; i < g->nf - 1; i++) F[IA(g) + i] = K->a[0] * un;"),
    "nu_wavespeed_width": ("(fabs(w[IU(&g) + d]) + cs) / cell_width(&g, d, (c / g.stride[d]) % g.n[d]);",
                           "(fabs(w[IU(&g) + d]) + cs) / g.dx[d];"),
    # the gated form's rule
    "gate_either_sensor": ("if (smooth_r && smooth_p) {", "if (smooth_r || smooth_p) {"),
    "gate_logit_sign": ("return *z < 0.0;", "return *z > 0.0;"),
    "gate_linear_weight": ("*vm = 0.1 * p0 + 0.6 * p1 + 0.3 * p2;", "*vm = 0.3 * p0 + 0.6 * p1 + 0.1 * p2;"),
    "gate_fallback_alpha": ("return rho > 0.0 && a1 >= 0.0 && a1 <= 1.0 && c > 0.0;", "return rho > 0.0 && c > 0.0;"),
    "gate_pressure_sensor": ("sp[s] = W5[s * neq + IE(g)];", "sp[s] = W5[s * neq + IU(g)];"),
    "gate_density_sensor": ("sr[s] = W5[s * neq + 0] + W5[s * neq + 1];", "sr[s] = W5[s * neq + 0];"),
}


# mistakes in the network's input normalisation (mlp_oracle.c)
MLP_MUTATIONS = {
    "gate_floor_ignored": ("if (!(m > delta * fabs(v5[2]))) {", "if (!(m > 0.0)) {"),
    "gate_norm_centre": ("x[k] = (v5[k] - v5[2]) / m;", "x[k] = (v5[k] - v5[0]) / m;"),
    "gate_norm_reversed": ("x[k] = (v5[k] - v5[2]) / m;", "x[k] = (v5[4 - k] - v5[2]) / m;"),
}


@pytest.mark.parametrize("name", sorted(MUTATIONS) + sorted(MLP_MUTATIONS))
def test_planted_mistake_is_caught(name, tmp_path):
    target = SRC if name in MUTATIONS else MLP_SRC
    before, after = MUTATIONS[name] if name in MUTATIONS else MLP_MUTATIONS[name]
    src = open(target).read()
    assert src.count(before) >= 1, "mutation anchor no longer in the oracle source"
    csrc = tmp_path / "mutant.c"
    csrc.write_text(src.replace(before, after))
    other = MLP_SRC if target == SRC else SRC
    so = tmp_path / "libmutant.so"
    subprocess.run(["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-o",
                    str(so), str(csrc), other, "-lm"], check=True)
    env = dict(os.environ, MFC5_ORACLE_LIB=str(so))
    suites = ["test_oracle_elements.py", "test_oracle_physics.py", "test_oracle_stretched.py",
              "test_oracle_nfluids.py", "test_oracle_gate.py", "test_oracle_mlp.py"]
    # the suite that pins the mutated part runs first (-x stops at the first
    # failing pin); every suite still runs for a mutant it does not catch
    first = {"gate": "test_oracle_gate.py", "nu": "test_oracle_stretched.py", "nf": "test_oracle_nfluids.py"}
    lead = first.get(name.split("_")[0])
    if lead:
        suites.remove(lead)
        suites.insert(0, lead)
    suites = [os.path.join(ROOT, "tests", f) for f in suites]
    r = subprocess.run([sys.executable, "-m", "pytest", *suites, "-x", "-q", "-p", "no:cacheprovider",
                        "-m", "not gpu"], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode != 0, f"mutation {name} passed every pin:\n{r.stdout[-2000:]}"
