"""GB300-native adaptive-force-update gravity path (Grudic 2020, Sections 2-3).

The compute path is the C-ABI library ``libgrav`` (hand-written CUDA for
sm_103a) reached through :mod:`paper_2010_13792_gb300.grav`.  Importing the
package is cheap; the library is loaded on first use and a missing or
unbuilt library raises instead of falling back to anything else.
"""
__all__ = ["grav", "ics"]
