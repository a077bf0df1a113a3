"""`python -m paper_1805_01407_gb300` builds libxr.so in place."""
from .build import build

print(build())
