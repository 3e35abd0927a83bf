"""The oracle's pins catch plausible mistakes (no GPU): each case plants one
mistake in a copy of oracle.cpp (a dropped term, a wrong sign, a transposed
operand or index, a flipped tie-break or threshold), builds it, and runs the
pin tests against that build; at least one pin must fail. The unmodified
oracle passes the same pins in the normal run. The phase of the Hopf grid's
fiber samples (psi_k = 2 pi (k + 1/2) / 6n) is a reading, not a fact of the
paper: a grid without the half step has the same fiber structure and
covering, which the pins check, so it is not planted here."""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "oracle.cpp")

ROT = ("  return {R[0] * p[0] + R[1] * p[1] + R[2] * p[2],\n"
       "          R[3] * p[0] + R[4] * p[1] + R[5] * p[2],\n"
       "          R[6] * p[0] + R[7] * p[1] + R[8] * p[2]};")
ROT_T = ("  return {R[0] * p[0] + R[3] * p[1] + R[6] * p[2],\n"
         "          R[1] * p[0] + R[4] * p[1] + R[7] * p[2],\n"
         "          R[2] * p[0] + R[5] * p[1] + R[8] * p[2]};")

# (name, text in oracle.cpp, planted replacement, occurrences)
MUTATIONS = [
    ("round_without_half", "v[0] = (Y[3 * j + 0] - u.x) / delta + 0.5;", "v[0] = (Y[3 * j + 0] - u.x) / delta;", 1),
    ("difference_sign", "v[1] = (Y[3 * j + 1] - u.y) / delta + 0.5;", "v[1] = (Y[3 * j + 1] + u.y) / delta + 0.5;", 1),
    ("transposed_rotation", ROT, ROT_T, 1),
    ("mode_ties_keep_larger_key", "if ((int64_t)(b - a) > best_len) {", "if ((int64_t)(b - a) >= best_len) {", 1),
    ("mode_index_decode", "kstar[1] = lo[1] + (int)((best_key / Ez) % Ey);",
     "kstar[1] = lo[1] + (int)((best_key / Ey) % Ez);", 1),
    ("lattice_box_floor", "lo[a] = (int)std::ceil((c[a] - s[a]) / delta);",
     "lo[a] = (int)std::floor((c[a] - s[a]) / delta);", 1),
    ("inlier_threshold_inclusive", "if (d[i] < eps) ++c;", "if (d[i] <= eps) ++c;", 1),
    ("q_filter_strict", "o[r].cand = 1000LL * o[r].M >= (int64_t)P->q_milli * Mstar;",
     "o[r].cand = 1000LL * o[r].M > (int64_t)P->q_milli * Mstar;", 1),
    ("top_k_ascending", "return o[a].M > o[b].M; });", "return o[a].M < o[b].M; });", 1),
    ("argmin_ties_keep_larger_index", "    return a < b;\n  };", "    return a > b;\n  };", 1),
    ("huber_without_half", "return e <= P->huber_h ? 0.5 * e * e :", "return e <= P->huber_h ? e * e :", 1),
    ("l1_not_truncated", "    case 1:  // truncated L1\n      return std::min(d, P->tau);",
     "    case 1:  // truncated L1\n      return d;", 1),
    ("euler_box_left_product", "matmul3(R0, Rz, T);", "matmul3(Rz, R0, T);", 1),
    ("refine_boxes_all_on_best", "const int64_t centre = cands[(size_t)std::min(c, nc - 1)];",
     "const int64_t centre = cands[0];", 1),
    ("nn_translation_sign", "const double qx = u.x + t[0], qy = u.y + t[1], qz = u.z + t[2];\n    double best",
     "const double qx = u.x - t[0], qy = u.y + t[1], qz = u.z + t[2];\n    double best", 1),
    ("refine_translation_sign", "const double qx = u.x + t[0], qy = u.y + t[1], qz = u.z + t[2];\n    double d1",
     "const double qx = u.x + t[0], qy = u.y - t[1], qz = u.z + t[2];\n    double d1", 1),
    ("nn_dropped_axis", "const double s = dx * dx + dy * dy + dz * dz;", "const double s = dx * dx + dy * dy;", 1),
    ("grid_voxel_corner_not_centre", "const double px = lo[0] + (a + 0.5) * h[0],", "const double px = lo[0] + a * h[0],", 1),
    ("grid_spacing_without_margin", "h[a] = (mx - mn + 2.0 * cap) / (double)(G - 2);",
     "h[a] = (mx - mn + 2.0 * cap) / (double)(G - 1);", 1),
    ("lookup_without_half_offset", "double g = (p[a] - lo[a]) / h[a] - 0.5;", "double g = (p[a] - lo[a]) / h[a];", 1),
    ("grid_not_capped", "D[((int64_t)a * G + b) * G + c] = std::min(cap, std::sqrt(best));",
     "D[((int64_t)a * G + b) * G + c] = std::sqrt(best);", 1),
    ("l2_not_squared", "      const double e = std::min(d, P->tau);\n      return e * e;",
     "      const double e = std::min(d, P->tau);\n      return e;", 1),
    ("lp_inverse_exponent", "return std::pow(d, P->p);", "return std::pow(d, 1.0 / P->p);", 1),
    ("inlier_metric_inclusive", "return d < P->epsilon ? 0.0 : 1.0;", "return d <= P->epsilon ? 0.0 : 1.0;", 1),
    ("exhaustive_inlier_inclusive", "if (d < P->epsilon) ++n_in;", "if (d <= P->epsilon) ++n_in;", 1),
    ("exhaustive_translation_sign", "const double dx = Y[3 * j] - u[3 * i] - t[0],",
     "const double dx = Y[3 * j] - u[3 * i] + t[0],", 1),
]


@pytest.mark.parametrize("name,old,new,count", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_pins_catch_planted_mistake(tmp_path, name, old, new, count):
    src = open(SRC).read()
    assert src.count(old) == count, f"{name}: mutation site not found as expected"
    mutant = tmp_path / "oracle_mutant.cpp"
    mutant.write_text(src.replace(old, new))
    lib = str(tmp_path / "liboracle_mutant.so")
    subprocess.check_call([shutil.which("g++") or "g++", "-O1", "-std=c++17", "-fPIC", "-shared", "-pthread", "-o",
                           lib, str(mutant)])
    env = dict(os.environ, DSES_ORACLE_LIB=lib)
    out = subprocess.run([sys.executable, "-m", "pytest", os.path.join(ROOT, "tests", "test_oracle_pins.py"), "-x",
                          "-q", "-p", "no:cacheprovider"], capture_output=True, text=True, timeout=600, cwd=ROOT,
                         env=env)
    assert out.returncode == 1, f"{name}: no pin failed\n{out.stdout[-1500:]}"
