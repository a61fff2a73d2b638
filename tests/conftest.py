import math
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

# Table I of the paper (Sec. IV-A): [d_s, d_min, d_ref] = [0.5, 0.5, 0.65],
# [theta_b, theta_s, theta_p] = [1.70, 0.36, 0.20], [c^B, alpha_d, alpha_b,
# alpha_s] = [50, 20, 20, 15].  The inflation distances are not in Table I;
# d_inf = 0.2 and d_sm = 0.4 are the values of the Fig. 3 caption.
PARAMS_TABLE1 = dict(d_min=0.5, d_ref=0.65, theta_b=1.70, theta_s=0.36, theta_p=0.20,
                     c_b=50.0, alpha_d=20.0, alpha_b=20.0, alpha_s=15.0,
                     d_inf=0.2, d_sm=0.4, patch_radius=2)

# The benchmark workloads' robot: height 0.5 m, maximum slope 30 deg
# (theta_s = tan 30 deg), inflation radius 0.3 m; the rest as Table I.
PARAMS_ROBOT = dict(PARAMS_TABLE1, theta_s=math.tan(math.radians(30.0)), d_inf=0.3, d_sm=0.4)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300) and the built libtct")


@pytest.fixture(scope="session")
def oracle_mod():
    import oracle
    oracle.compile_library()
    return oracle
