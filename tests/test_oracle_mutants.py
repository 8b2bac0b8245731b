"""Planted mistakes: each mutant is a copy of the oracle source with one
plausible error (a dropped term, a wrong sign, a transposed operand, a wrong
index).  The pins must reject every one of them.  CPU only; the mutants are
compiled into a temporary directory and never touch the real oracle build."""
import concurrent.futures as cf
import os
import subprocess
import tempfile

import pytest

from oracle import oracle as orc
from tests import test_oracle_pins as pins

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle", "rr_oracle.c")

MUTANTS = {
    "philox_multiplier": ("0xD2511F53u", "0xD2511F54u"),
    "u24_bits": ("(2u * (x >> 9) + 1u)", "(2u * (x >> 8) + 1u)"),
    "box_muller_scale": ("sqrt(-2.0 * log(u0))", "sqrt(-log(u0))"),
    "d3_half_width": ("0.5 * beam_width / (sqrt(2.0) * orc_erfinv(beam_prob))",
                      "beam_width / (sqrt(2.0) * orc_erfinv(beam_prob))"),
    "fresnel_drop_p": ("*R = 0.5 * (rs * rs + rp * rp);", "*R = rs * rs;"),
    "fresnel_transposed": ("double rp = (n1 * ct - n2 * cos_i) / (n1 * ct + n2 * cos_i);",
                           "double rp = (n1 * cos_i - n2 * ct) / (n1 * ct + n2 * cos_i);"),
    "snell_inverted": ("  double eta = n1 / n2;\n  double sin2_t", "  double eta = n2 / n1;\n  double sin2_t"),
    "reflect_sign": ("out[i] = d[i] - 2.0 * dn * n[i];", "out[i] = d[i] + 2.0 * dn * n[i];"),
    "refract_sign": ("(eta * cos_i - cos_t) * n[i]", "(eta * cos_i + cos_t) * n[i]"),
    "brdf_norm_drop_B": ("return m->A * M_PI + 2.0 * m->B + S * sqrt(M_PI) * gr;",
                         "return m->A * M_PI + S * sqrt(M_PI) * gr;"),
    "brdf_window_B_term": ("m->B * (sin(hi) - sin(lo))", "m->B * (cos(lo) - cos(hi))"),
    "traveled_angle": ("window(s, mid, 2.0 * theta0, b)", "window(s, mid, theta0, b)"),
    "attenuation_factor": ("exp(-2.0 * alpha_np(", "exp(-alpha_np("),
    "geometric_range": ("double L1 = ray.L + n_cur * h.t;", "double L1 = ray.L + h.t;"),
    "air_range_half": ("range_a = 0.5 * (L1 + dist);", "range_a = L1 + dist;"),
    "mt_operand": ("*b2 = dot3(d, qv) * inv;", "*b2 = dot3(tv, qv) * inv;"),
    "blur_clamp_edges": ("if (src < 0 || src >= (long)nb) continue;",
                         "if (src < 0) src = 0;\n          if (src >= (long)nb) src = nb - 1;"),
    "no_depletion": ("double e_refl = E1 * R - ret_t - (air_uses_T ? 0.0 : ret_a);", "double e_refl = E1 * R;"),
    "receive_weight": ("exp(-0.5 * delta * delta * f / (sigma * sigma))", "exp(-delta * delta * f / (sigma * sigma))"),
    "noise_same_uniform": ("va = orc_u24(xa[0]);", "va = orc_u24(xs[0]);"),
    "elliptic_ignored": ("double th = p->elevation + p->beam_aspect * r * sin(omega);",
                         "double th = p->elevation + r * sin(omega);"),
    "elliptic_weight_inverted": ("ce * ce / (p->beam_aspect * p->beam_aspect)",
                                 "ce * ce * (p->beam_aspect * p->beam_aspect)"),
    "perlin_smoothstep": ("return t * t * t * (t * (6.0 * t - 15.0) + 10.0);", "return t * t * (3.0 - 2.0 * t);"),
    "perlin_corner_swap": ("perlin_grad(p, i1, j0, purpose, g10);", "perlin_grad(p, i0, j1, purpose, g10);"),
    "perlin_not_periodic": ("i1 = (i0 + 1u) % (uint32_t)P;", "i1 = i0 + 1u;"),
    "perlin_scale": ("return 0.5 + n / sqrt(2.0);", "return 0.5 + n;"),
    "ct_diffuse_norm": ("return m->A * 0.5 * cos(w)", "return m->A * cos(w)"),
    "ct_half_angle": ("orc_beckmann(0.5 * w, m->B)", "orc_beckmann(w, m->B)"),
    "beckmann_norm_term": ("(1.0 + 0.5 * m * m)", "(1.0 + m * m)"),
    "table_prim_coeff": ("f0 * (s3 / 6.0 - 0.75 * s2 + s)", "f0 * (s3 / 6.0 - 0.5 * s2 + s)"),
    "table_symmetry": ("return table_prim(t, hi) + table_prim(t, -lo);",
                       "return table_prim(t, hi) - table_prim(t, -lo);"),
    "air_side": ("          if (side <= 0.0) candidate = 0;", "          if (side >= 0.0) candidate = 0;"),
    "traveled_range_half": ("push_ret(col, k, L1, e);", "push_ret(col, k, 0.5 * L1, e);"),
    "bin_off_by_one": ("img[(size_t)fb] += r->E;", "img[(size_t)fb + 1] += r->E;"),
    "index_is_permittivity": ("    n2 = sqrt(m->eps_r);", "    n2 = m->eps_r;"),
    "reflected_child_medium": ("        c.medium = ray.medium;", "        c.medium = next_medium;"),
    "speckle_mean_two": ("return -log(orc_u24(x[which]));", "return 1.0 - log(orc_u24(x[which]));"),
    "speckle_shared_word": ("orc_speckle_factor(p, a, k, ray.path, ray.bounce, 1)",
                            "orc_speckle_factor(p, a, k, ray.path, ray.bounce, 0)"),
    "speckle_counter_swapped": ("draw(p, a, k, 1u | (((path << 8) | bounce) << 8), x);",
                                "draw(p, a, k, 1u | (((bounce << 8) | path) << 8), x);"),
    "min_energy_doubled": ("int spawn_refl = deeper && in_range && e_refl >= p->min_energy;",
                           "int spawn_refl = deeper && in_range && e_refl >= 2.0 * p->min_energy;"),
    "range_weight_round_trip": ("return pow(r, -p->range_falloff);", "return pow(2.0 * r, -p->range_falloff);"),
    "azimuth_step": ("double phi = 2.0 * M_PI * (double)a / (double)p->n_azimuth + r * cos(omega);",
                     "double phi = M_PI * (double)a / (double)p->n_azimuth + r * cos(omega);"),
}

CHECKS = [c for c in pins.ALL_CHECKS] + [lambda: pins.check_d3_statistics(4000)]


@pytest.fixture(scope="module")
def mutant_libs():
    src = open(SRC).read()
    tmp = tempfile.mkdtemp(prefix="oracle_mutants_")

    def build(item):
        name, (old, new) = item
        assert src.count(old) == 1, f"mutation site for {name} not unique"
        path = os.path.join(tmp, f"{name}.c")
        with open(path, "w") as f:
            f.write(src.replace(old, new))
        so = os.path.join(tmp, f"lib_{name}.so")
        subprocess.run(["gcc", "-O1", "-std=gnu11", "-shared", "-fPIC", "-o", so, path, "-lm"], check=True,
                       capture_output=True)
        return name, so

    with cf.ThreadPoolExecutor(max_workers=os.cpu_count() or 4) as ex:
        libs = dict(ex.map(build, MUTANTS.items()))
    return libs


@pytest.mark.slow
@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(mutant_libs, name):
    prev = orc.use_library(mutant_libs[name])
    caught = []
    try:
        for check in CHECKS:
            try:
                check()
            except Exception as e:  # noqa: BLE001 -- any failure counts as caught
                caught.append(getattr(check, "__name__", "d3_statistics"))
                break
    finally:
        orc.restore_library(prev)
    assert caught, f"no pin rejects the planted mistake {name}"
