"""The single-precision walk's material-lookup program, as the host chooses it.

The one-shape programs count steps by region (earth side of the surface,
inside the shape) and turn the counts into material counts at the walk's
exit (the occupation update of Sec. 3.1).  That is right only for a shape
that lies wholly on one side of the surface z = 0, so the host must send any
other shape to the general program.  sdd_model_program runs the same host
decision without a GPU.
"""
import pytest

from paper_1603_09311_gb300 import build as B
from paper_1603_09311_gb300 import inputs as I
from paper_1603_09311_gb300 import sdd


@pytest.fixture(scope="module", autouse=True)
def built():
    B.build()
    sdd.lib()


def _one(kind, v):
    return {"domain": I.DOMAIN, "kappa": [[0.0, 2.0, 20.0]], "bg": (0, 1),
            "shapes": [(kind, 2, tuple(v))], "g": ("columns", 1, 1)}


def _rect(x0, x1, z0, z1):
    return _one(0, (x0, x1, z0, z1, 0.0, 0.0))


def _tri(*pts):
    return _one(1, tuple(c for p in pts for c in p))


@pytest.mark.parametrize("model,program,side", [
    (I.halfspace(2.0), "layers", -1),
    (I.quarterspace(2.0, 20.0), "contact", 0),
    (I.block_batched(), "rect", 0),
    (I.triangle(), "triangle", 0),
    (_rect(-0.3, 0.3, -0.4, -0.1), "rect", 1),
    # a rectangle whose bottom is the surface is in the earth (half-open in z),
    # one whose top is the surface is in the air
    (_rect(-0.3, 0.3, 0.0, 0.4), "rect", 0),
    (_rect(-0.3, 0.3, -0.4, 0.0), "rect", 1),
    (_rect(-0.2, 0.3, -0.2, 0.3), "shapes4", -1),
    (_tri((-0.4, -0.45), (0.3, -0.35), (-0.1, -0.05)), "triangle", 1),
    # a vertex on the surface, or just above it within the FP32 test's
    # rounding, is not far enough from it: the general program
    (_tri((-0.3, 0.2), (0.3, 0.2), (0.0, 0.0)), "shapes4", -1),
    (_tri((-0.3, 0.2), (0.3, 0.2), (0.0, 1e-8)), "shapes4", -1),
    (_tri((-0.3, 0.2), (0.3, 0.2), (0.0, 1e-3)), "triangle", 0),
    (_tri((-0.3, 0.2), (0.3, 0.2), (0.0, -0.1)), "shapes4", -1),
])
def test_one_shape_programs_only_for_a_shape_on_one_side(model, program, side):
    assert sdd.sdd_model_program(model) == (program, side)


def test_other_programs():
    two = I.quarterspace(2.0, 20.0)
    two["shapes"] = two["shapes"] + [(0, 1, (-0.5, -0.2, 0.1, 0.3, 0.0, 0.0))]
    assert sdd.sdd_model_program(two) == ("shapes4", -1)
    many = dict(two)
    many["shapes"] = [(0, 2, (-0.9 + 0.3 * k, -0.8 + 0.3 * k, 0.1, 0.3, 0.0, 0.0)) for k in range(5)]
    assert sdd.sdd_model_program(many) == ("shapes16", -1)
    r = I.triangle()
    r["raster"] = I.rasterize(r)
    r["shapes"] = []
    assert sdd.sdd_model_program(r) == ("raster", -1)
    assert sdd.sdd_model_program(I.tm_analytic()) == ("tm", -1)


def test_a_bad_model_is_rejected():
    m = I.halfspace(2.0)
    m["kappa"] = [[0.0, -1.0]]
    with pytest.raises(sdd.SddError) as e:
        sdd.sdd_model_program(m)
    assert e.value.status == sdd.SDD_E_ARG
