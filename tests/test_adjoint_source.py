"""Source guard for the adjoint kernel (csrc/adjoint_kernels.cuh).

Adjoint::substep() runs the stage loop of one RK4 substep as a rolled loop.
With two inlined copies of that loop in run(), the compiled kernels (nvcc 13.0,
sm_103a) gave wrong velocity gradients although the source forms are
equivalent; with one call site they pass every parity test.  This CPU test
keeps the call site single, so that the hazard cannot come back unnoticed
before the GPU parity tests run."""
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
ADJOINT = os.path.join(ROOT, "paper_2103_02388_gb300", "csrc", "adjoint_kernels.cuh")


def _code(path):
    """Source without comments."""
    with open(path) as f:
        src = f.read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return re.sub(r"//[^\n]*", "", src)


def test_substep_has_one_call_site():
    code = _code(ADJOINT)
    definitions = re.findall(r"__device__\s+void\s+substep\s*\(", code)
    uses = re.findall(r"\bsubstep\s*\(", code)
    assert len(definitions) == 1
    assert len(uses) - len(definitions) == 1, "substep() must keep a single call site"
