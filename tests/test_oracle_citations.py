"""Every public function and class of the oracle names the passage of the paper it follows
(a section, an equation, a table or an algorithm), the reading it takes where the paper is
silent, or says that it has no counterpart in the paper (the selector).  Every module's header
says that it is test infrastructure."""
import ast
import os
import re

import pytest

ORACLE = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle")
CITES = re.compile(r"Secs?\.|Eqs?\.|Table|Algorithm|counterpart|[Rr]eading")


def _public(path):
    tree = ast.parse(open(path).read())
    for node in tree.body:
        if isinstance(node, (ast.FunctionDef, ast.ClassDef)) and not node.name.startswith("_"):
            yield node.name, ast.get_docstring(node) or ""


@pytest.mark.parametrize("module", sorted(f for f in os.listdir(ORACLE) if f.endswith(".py")))
def test_every_public_oracle_function_cites_its_passage(module):
    path = os.path.join(ORACLE, module)
    missing = [name for name, doc in _public(path) if not CITES.search(doc)]
    assert not missing, f"{module}: {missing}"
    head = " ".join((ast.get_docstring(ast.parse(open(path).read())) or "").lower().split())
    assert "test infrastructure" in head, f"{module}: the header does not say it is test infrastructure"
