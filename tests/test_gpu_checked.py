"""The checked build (libpifcm_checked.so, -DIFCM_CHECKED) on the odd shapes
of the parity suite: every computed global index of the stencil, plain and
reduce kernels (membership stores, partial-record writes and reads, TMA plane
coordinates, the item table) is tested against its buffer before the access,
and a violation would record IFCM_ERR_BOUNDS in the status word.  Each case
must finish with status OK and match the FP64 oracle.  The library is loaded
in a child process so that it does not replace the normal build of this
test session."""
import json
import os
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r'''
import json, sys
sys.path.insert(0, ROOT)
import numpy as np, torch
from paper_2002_01981_gb300 import build, native
native.load(build.CHECKED_LIB_PATH)
from paper_2002_01981_gb300 import ifcm as G, phantoms
G.resident_enable(False)      # the stencil kernels on every shape
from oracle import ifcm as O
from oracle import pso as OP

def dev(a):
    return torch.from_numpy(phantoms.pad_pitch(np.asarray(a, np.float32))).cuda()

def dev_u(u):
    c, nz, ny, nx = u.shape
    out = np.zeros((c, nz, ny, phantoms.pitch_for(nx)), np.float32)
    out[..., :nx] = u
    return torch.from_numpy(out).cuda()

out = []
for shape, c in [((1, 1, 1), 2), ((1, 1, 7), 3), ((2, 2, 2), 5), ((5, 17, 70), 3),
                 ((37, 30, 70), 4), ((1, 100, 45), 4), ((9, 14, 21), 6)]:
    nz, ny, nx = shape
    x = np.clip(phantoms.brain_phantom(shape, seed=5, sigma=0.06), 0, 1).astype(np.float32)
    U = phantoms.random_memberships(shape, c, seed=6)
    C = np.linspace(0.15, 0.85, c)
    lx = np.array([[0.4, 0.3], [0.7, 0.2], [0.1, 0.6]])
    it = 4
    prm = G.Params(c=c, max_iter=it, eps_u=0.0)
    r = {"shape": shape, "c": c}
    # one particle (planar layout)
    Ug, _, Jg, _ = G.ifcm_fit(dev(x), prm, (0.4, 0.3), nx=nx, u_init=dev_u(U), c_init=C)
    Uo, _, Jo, _ = O.ifcm_fit(x.astype(np.float64), U.astype(np.float64), C, 0.4, 0.3, 2.0,
                              it, 0.0)
    r["fit_u"] = float(np.max(np.abs(Ug[..., :nx].cpu().numpy() - Uo)))
    # three particles (float2 pair words; 3D iterations after the first on
    # the leaner kernel), then bf16 pair words
    fo, _ = OP.fitness_batch(x.astype(np.float64), U.astype(np.float64), C, lx, max_iter=it,
                             eps=0.0)
    fg, _, _ = G.pso_fitness_batch(dev(x), prm, lx, dev_u(U), C, nx=nx)
    r["batch_j"] = float(np.max(np.abs(fg.cpu().numpy() - fo) / np.abs(fo)))
    fb, _, _ = G.pso_fitness_batch(dev(x), G.Params(c=c, max_iter=it, eps_u=0.0, u_dtype="bf16"),
                                   lx, dev_u(U), C, nx=nx)
    r["bf16_j"] = float(np.max(np.abs(fb.cpu().numpy() - fo) / np.abs(fo)))
    # the plain form and Eq 10 shells (V = 2)
    Up, _, _, _ = G.ifcm_fit(dev(x), prm, (0.4, 0.3), nx=nx, u_init=dev_u(U), c_init=C,
                             plain=True)
    r["plain_u"] = float(np.max(np.abs(Up[..., :nx].cpu().numpy() - Uo)))
    fs, _, _ = G.pso_fitness_batch(dev(x), G.Params(c=c, V=2, max_iter=2, eps_u=0.0), lx,
                                   dev_u(U), C, nx=nx)
    fso, _ = OP.fitness_batch(x.astype(np.float64), U.astype(np.float64), C, lx, max_iter=2,
                              eps=0.0, V=2)
    r["shell_j"] = float(np.max(np.abs(fs.cpu().numpy() - fso) / np.abs(fso)))
    out.append(r)
print("RESULT " + json.dumps(out))
'''


def test_checked_build_on_odd_shapes():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2002_01981_gb300 import build
    build.build(checked=True)
    env = dict(os.environ)
    r = subprocess.run([sys.executable, "-c", CHILD.replace("ROOT", repr(ROOT), 1)],
                       capture_output=True, text=True, timeout=900, env=env, cwd=ROOT)
    # a status other than OK (IFCM_ERR_BOUNDS above all) raises in the child
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    line = [ln for ln in r.stdout.splitlines() if ln.startswith("RESULT ")][-1]
    for case in json.loads(line[len("RESULT "):]):
        assert case["fit_u"] <= 1e-5, case
        assert case["plain_u"] <= 1e-5, case
        assert case["batch_j"] <= 1e-5, case
        assert case["shell_j"] <= 1e-5, case
        assert case["bf16_j"] <= 1e-2, case
