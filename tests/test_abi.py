"""The C-ABI library loads, exports every entry point declared in include/mlvs.h, and rejects
bad configurations on the host before touching a device."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "mlvs.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(mlvs_[a-z_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    from paper_2609_35258_b300 import mlvs
    lib = ctypes.CDLL(mlvs._LIB_PATH)
    names = _declared()
    assert "mlvs_create" in names and "mlvs_step" in names
    for n in names:
        assert hasattr(lib, n), n


def test_python_binding_names_match_header():
    from paper_2609_35258_b300 import mlvs
    for n in _declared():
        assert callable(getattr(mlvs, n)), n


def _cfg(**kw):
    from paper_2609_35258_b300 import mlvs
    W = np.zeros((1, 4, 4, 4))
    W[..., 0] = 1.0
    W[..., 3] = 1.0
    args = dict(dim=2, nx=4, ny=4, Lx=1.0, Ly=1.0, bc=[0, 0, 0, 0], init_W=W, Kn=0.1)
    args.update(kw)
    return mlvs.make_config(**args)


@pytest.mark.parametrize("bad", [dict(dim=3), dict(nx=0), dict(bc=[0, 2, 0, 0]),
                                 dict(Kn=0.0, mu_ref=0.0), dict(storage=7), dict(dim=1, ny=4),
                                 dict(map_moments=8), dict(positive_mapping=2)])
def test_create_rejects_bad_config(bad):
    from paper_2609_35258_b300 import mlvs
    with pytest.raises(mlvs.MLVSError) as e:
        mlvs.mlvs_create(_cfg(**bad))
    assert e.value.status == -1
    assert mlvs.mlvs_last_error(None)


def test_create_rejects_nonpositive_state():
    from paper_2609_35258_b300 import mlvs
    W = np.zeros((1, 4, 4, 4))
    W[..., 0] = 1.0      # T = 0
    with pytest.raises(mlvs.MLVSError):
        mlvs.mlvs_create(_cfg(init_W=W))


def test_destroy_null_is_safe():
    from paper_2609_35258_b300 import mlvs
    mlvs.mlvs_destroy(None)


def test_every_entry_point_cites_its_passage_or_says_it_has_none():
    """Each declaration's comment names the section or equation it implements, or says that the
    paper has no counterpart (utilities, the selector, the allocation-free variant)."""
    src = open(os.path.join(ROOT, "include", "mlvs.h")).read()
    missing = []
    for m in re.finditer(r"/\*((?:(?!\*/).)*)\*/\s*(?:enum\s*\{[^}]*\};\s*/\*((?:(?!\*/).)*)\*/\s*)?"
                         r"(?:const\s+)?(?:mlvs_status|void|const char\s*\*)\s*\*?\s*(mlvs_[a-z_]+)\s*\(", src, re.S):
        com = m.group(2) or m.group(1)
        if not re.search(r"Sec\.|Eqs?\.|counterpart|Not part of the paper", com):
            missing.append(m.group(3))
    assert not missing, missing
