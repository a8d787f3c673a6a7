"""Seeded synthetic inputs (volumes and cameras) shared by the tests, the
benchmark and the oracle checks.  No part of the rendering method lives here."""
from . import cameras, volumes  # noqa: F401
