"""The entry point the round-end check runs on a GPU: one small synthesis and
round trip per form, checked against the oracle inside smoke() itself."""
import pytest

pytestmark = pytest.mark.gpu


def test_graft_entry_smoke():
    torch = pytest.importorskip("torch")
    assert torch.cuda.is_available()
    import __graft_entry__

    __graft_entry__.build()
    __graft_entry__.smoke()
